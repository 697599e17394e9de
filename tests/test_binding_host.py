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


class FakeHandleLib:
    """Stand-in for the library: a handle with W walkers that records calls."""

    def __init__(self, W):
        self.W, self.calls = W, []

    def qmc_n_walkers(self, h):
        return self.W

    def __getattr__(self, name):
        def call(*a):
            self.calls.append((name,) + a)
            return 0
        return call


@pytest.fixture
def handle(monkeypatch):
    f = FakeHandleLib(W=6)
    monkeypatch.setattr(Q, "lib", lambda: f)
    return f


def test_per_walker_buffers_of_the_right_size_pass(handle):
    W, N = 6, 4
    Q.qmc_evaluate(None, np.zeros(W), np.zeros(W), np.zeros(W), np.zeros((W, N, 3)))
    Q.qmc_eval_cached(None, np.zeros(W), None, np.zeros(W), None)
    Q.qmc_force_vjp(None, np.zeros(W), np.zeros(W), np.zeros((3, 3)), None)
    Q.qmc_vmc(None, 5, 0.1, 0, np.zeros((5, W)))
    Q.qmc_force_estimate(None, np.ones(W), np.zeros((3, 3)))
    Q.qmc_get_walkers(None, np.zeros((W, N, 3)), np.zeros(W))
    Q.qmc_jastrow_derivs(None, np.zeros((W, 7)), np.zeros((W, 7)))
    Q.qmc_set_walkers(None, np.zeros((W, N, 3), dtype=np.float32))   # host arrays are converted
    names = [c[0] for c in handle.calls]
    assert names == ["qmc_evaluate", "qmc_eval_cached", "qmc_force_vjp", "qmc_vmc", "qmc_force_estimate",
                     "qmc_get_walkers", "qmc_jastrow_derivs", "qmc_set_walkers"]


@pytest.mark.parametrize("case", ["short eloc", "float32 eloc", "short trace", "short weights", "int32 grad",
                                  "float32 tensor walkers", "short g_eloc"])
def test_short_or_mistyped_buffers_are_refused(handle, case):
    W, N = 6, 4
    with pytest.raises(ValueError):
        if case == "short eloc":
            Q.qmc_evaluate(None, None, None, np.zeros(W - 1), None)
        elif case == "float32 eloc":
            Q.qmc_eval_cached(None, None, None, np.zeros(W, dtype=np.float32), None)
        elif case == "short trace":
            Q.qmc_vmc(None, 5, 0.1, 0, np.zeros((4, W)))
        elif case == "short weights":
            Q.qmc_force_estimate(None, np.ones(W - 2), np.zeros((3, 3)))
        elif case == "int32 grad":
            Q.qmc_evaluate(None, None, None, None, np.zeros((W, N, 3), dtype=np.int32))
        elif case == "float32 tensor walkers":
            Q.qmc_set_walkers(None, torch.zeros((W, N, 3), dtype=torch.float32))
        else:
            Q.qmc_force_vjp(None, np.zeros(W - 1), None, np.zeros((3, 3)), None)
    assert not handle.calls
