"""Argument checks of the Python binding's tensor-core GEMM entry points, on
the host: the shapes the GPU tests and smoke() use are accepted and reach
the C call with the strides they had; mismatched shapes, host tensors and
non-contiguous arrays are refused before any library call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2504_07948_gb300 import qmc as Q


class FakeLib:
    def __init__(self):
        self.calls = []

    def qmc_tc_gemm(self, *a):
        self.calls.append(("gemm",) + a)
        return 0

    def qmc_tc_gemm_split(self, *a):
        self.calls.append(("split",) + a)
        return 0


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(Q, "lib", lambda: f)
    monkeypatch.setattr(Q, "_need_f32_cuda", lambda *ts: None)   # host tensors stand in for device ones
    return f


@pytest.mark.parametrize("batch,M,N,K,share_a,b_trans", [
    (3, 200, 48, 40, False, False), (4, 300, 160, 160, True, False), (2, 160, 160, 160, False, True),
    (2, 50, 250, 33, False, True), (3, 257, 96, 100, True, True), (2, 130, 32, 24, False, False)])
def test_gemm_shapes_of_the_tests_are_accepted(fake, batch, M, N, K, share_a, b_trans):
    A = torch.zeros((1 if share_a else batch, M, K))
    B = torch.zeros((batch, K, N) if b_trans else (batch, N, K))
    D = torch.zeros((batch, M, N))
    Q.qmc_tc_gemm(A, B, D, b_trans=b_trans)
    c = fake.calls[-1]
    assert c[1:5] == (batch, M, N, K)
    assert c[6] == (0 if share_a else M * K) and c[7] == K
    assert c[9] == B.shape[1] * B.shape[2] and c[10] == (N if b_trans else K) and c[11] == int(b_trans)
    assert c[13] == M * N and c[14] == N


@pytest.mark.parametrize("bad", ["A rows", "B cols", "A batch", "2-D"])
def test_gemm_mismatched_shapes_are_refused(fake, bad):
    A, B, D = torch.zeros((2, 8, 4)), torch.zeros((2, 16, 4)), torch.zeros((2, 8, 16))
    if bad == "A rows":
        A = torch.zeros((2, 9, 4))
    elif bad == "B cols":
        B = torch.zeros((2, 16, 5))
    elif bad == "A batch":
        A = torch.zeros((3, 8, 4))
    else:
        D = torch.zeros((8, 16))
    with pytest.raises(ValueError):
        Q.qmc_tc_gemm(A, B, D)
    assert not fake.calls


def test_split_shapes(fake):
    Q.qmc_tc_gemm_split(torch.zeros(7, 32), torch.zeros(7, 32), torch.zeros(16, 32), torch.zeros(16, 32),
                        torch.zeros(7, 16))
    assert fake.calls[-1][1:4] == (7, 16, 32)
    with pytest.raises(ValueError):
        Q.qmc_tc_gemm_split(torch.zeros(7, 32), torch.zeros(7, 31), torch.zeros(16, 32), torch.zeros(16, 32),
                            torch.zeros(7, 16))
    with pytest.raises(ValueError):
        Q.qmc_tc_gemm_split(torch.zeros(7, 32), torch.zeros(7, 32), torch.zeros(16, 32), torch.zeros(16, 32),
                            torch.zeros(16, 7))


def test_host_tensors_and_strided_arrays_are_refused():
    with pytest.raises(ValueError):
        Q.qmc_tc_gemm(torch.zeros(1, 4, 4), torch.zeros(1, 4, 4), torch.zeros(1, 4, 4))
    with pytest.raises(ValueError):
        Q._ptr(np.zeros((4, 4))[:, ::2])
