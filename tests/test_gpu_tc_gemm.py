"""Tensor-core (tcgen05, 3xTF32) batched GEMM of the mixed force path against
an FP64 product of the same FP32 inputs, through the C ABI.

Bound: |D - D_ref| <= 4e-6 sum_k |A_mk B_nk| per element: the 3xTF32 split
drops the lo*lo product (relative 2^-22) and accumulates in FP32 (K roundings
of 2^-24), far below the O(1) errors of a wrong tile layout or descriptor.
Shapes span ragged row tiles, ragged K stages, N from 16 to 256, shared and
per-batch operands and the transposed-B form the force path uses; operands
TMA can describe (16-byte aligned rows) take the pipelined kernel, the rest
(odd K) the staged one.
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
    (1, 5000, 160, 768, False, False),  # basis -> orbital shape (5 components x walkers, N_b = 768)
    (3, 257, 96, 100, True, True),      # shared A, transposed B, ragged K and rows
    (2, 130, 24, 1000, False, False),   # long K (63 stages of the pipelined kernel)
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


def tf32_round(x):
    """Round float32 values to the nearest TF32 value (10 mantissa bits),
    ties away from zero, as integer arithmetic on the bit patterns."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return r.view(np.float32)


@pytest.mark.parametrize("M,N,K", [(5000, 160, 768), (300, 32, 160), (130, 256, 96), (7, 16, 32), (260, 40, 100)])
def test_tc_gemm_split_matches_fp64(env, M, N, K):
    """Pre-split operands (hi = TF32(x), lo = TF32(x - hi)) through the
    swizzled TMA kernel: the product of the halves against FP64, at the
    3xTF32 bound; K = 100 leaves a ragged last stage, M = 7 a ragged tile."""
    torch, Q = env
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(N, K)).astype(np.float32)
    Ah = tf32_round(A)
    Al = tf32_round(A - Ah)
    Bh = tf32_round(B)
    Bl = tf32_round(B - Bh)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    Q.qmc_tc_gemm_split(dev(Ah), dev(Al), dev(Bh), dev(Bl), D)
    torch.cuda.synchronize()
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
    rel = float((np.abs(D.cpu().numpy().astype(np.float64) - ref) / scale).max())
    assert rel < 4e-6, rel
