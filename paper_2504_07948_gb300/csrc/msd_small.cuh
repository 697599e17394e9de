// Cofactors of the small (e <= 4) minors of the multi-determinant table.
#pragma once

namespace qmc {

// Cofactors of the leading e x e block of m: cof[a][c] = (-1)^(a+c) times
// the minor without row a and column c, i.e. det(m with column c replaced by
// the unit vector e_a).  Entries outside the block are zero.
template <typename F>
__device__ __forceinline__ void cofactors(int e, const F m[4][4], F cof[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) cof[a][c] = F(0);
    if (e == 1) {
        cof[0][0] = F(1);
    } else if (e == 2) {
        cof[0][0] = m[1][1];
        cof[0][1] = -m[1][0];
        cof[1][0] = -m[0][1];
        cof[1][1] = m[0][0];
    } else if (e == 3) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int r0 = a == 0 ? 1 : 0, r1 = a == 2 ? 1 : 2;
                const int c0 = c == 0 ? 1 : 0, c1 = c == 2 ? 1 : 2;
                const F mn = m[r0][c0] * m[r1][c1] - m[r0][c1] * m[r1][c0];
                cof[a][c] = ((a + c) & 1) ? -mn : mn;
            }
    } else if (e == 4) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int r0 = a == 0 ? 1 : 0, r1 = a <= 1 ? 2 : 1, r2 = a == 3 ? 2 : 3;
                const int c0 = c == 0 ? 1 : 0, c1 = c <= 1 ? 2 : 1, c2 = c == 3 ? 2 : 3;
                const F mn = m[r0][c0] * (m[r1][c1] * m[r2][c2] - m[r1][c2] * m[r2][c1]) -
                             m[r0][c1] * (m[r1][c0] * m[r2][c2] - m[r1][c2] * m[r2][c0]) +
                             m[r0][c2] * (m[r1][c0] * m[r2][c1] - m[r1][c1] * m[r2][c0]);
                cof[a][c] = ((a + c) & 1) ? -mn : mn;
            }
    }
}

}  // namespace qmc
