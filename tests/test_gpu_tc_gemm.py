"""Tensor-core (tcgen05, 3xTF32) batched GEMM of the mixed force path against
an FP64 product of the same FP32 inputs, through the C ABI.

Bound: |D - D_ref| <= 4e-6 sum_k |A_mk B_nk| per element: the 3xTF32 split
drops the lo*lo product (relative 2^-22) and accumulates in FP32 (K roundings
of 2^-24), far below the O(1) errors of a wrong tile layout or descriptor.
Shapes span ragged row tiles, ragged K stages, N from 16 to 256, shared and
per-batch operands and the transposed-B form the force path uses.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_07948_gb300 import qmc
    return torch, qmc


def run_case(env, batch, M, N, K, share_a=False, b_trans=False, seed=0):
    torch, Q = env
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(1 if share_a else batch, M, K)).astype(np.float32)
    B = rng.normal(size=(batch, K, N) if b_trans else (batch, N, K)).astype(np.float32)
    D = torch.full((batch, M, N), float("nan"), dtype=torch.float32, device="cuda")
    Q.qmc_tc_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), D, b_trans=b_trans)
    torch.cuda.synchronize()
    A64 = np.broadcast_to(A.astype(np.float64), (batch, M, K))
    Bt = B.astype(np.float64) if b_trans else np.transpose(B.astype(np.float64), (0, 2, 1))
    ref = A64 @ Bt
    scale = np.abs(A64) @ np.abs(Bt)
    err = np.abs(D.cpu().numpy().astype(np.float64) - ref)
    return float((err / np.maximum(scale, 1e-30)).max())


@pytest.mark.parametrize("batch,M,N,K,share_a,b_trans", [
    (3, 200, 48, 40, False, False),     # two row tiles (second ragged), ragged K stage
    (4, 300, 160, 160, True, False),    # shared A (coefficients), N = n of the 32-water cluster
    (2, 160, 160, 160, False, True),    # B given as [K][N] (Q = PT AT)
    (1, 128, 256, 64, False, False),    # widest accumulator
    (2, 7, 16, 8, False, False),        # smallest tile
    (2, 50, 250, 33, False, True),      # N padded to 256, odd K
])
def test_tc_gemm_matches_fp64(env, batch, M, N, K, share_a, b_trans):
    rel = run_case(env, batch, M, N, K, share_a, b_trans)
    assert rel < 4e-6, rel


def test_tc_gemm_zero_k_and_bad_sizes(env):
    torch, Q = env
    D = torch.full((2, 5, 16), 7.0, dtype=torch.float32, device="cuda")
    A = torch.zeros((2, 5, 1), dtype=torch.float32, device="cuda")
    B = torch.zeros((2, 16, 1), dtype=torch.float32, device="cuda")
    st = Q.lib().qmc_tc_gemm(2, 5, 16, 0, A.data_ptr(), 5, 1, B.data_ptr(), 16, 1, 0, D.data_ptr(), 80, 16, None)
    assert st == 0 and float(D.abs().max()) == 0.0
    st = Q.lib().qmc_tc_gemm(1, 5, 300, 4, A.data_ptr(), 0, 4, B.data_ptr(), 0, 4, 0, D.data_ptr(), 0, 300, None)
    assert st == -1   # N above 256
