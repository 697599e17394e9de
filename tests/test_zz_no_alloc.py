"""Allocation-free branching (qmc_branch_noalloc) against the DMC step of
the handle-based API.

Some callers cannot allocate device memory: they own every device buffer
and hand the library pointers only.  qmc_branch_noalloc serves them with its
scratch in a fixed device array.  Here it must reproduce, from the same
energies and random stream, the population that qmc_dmc produced, on two
calls in a row (the second call reuses the scratch the first one left).
"""
import numpy as np
import pytest

from paper_2504_07948_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_07948_gb300 import qmc
    return qmc


def test_branch_noalloc_matches_dmc_step(Q):
    import torch
    s = synth.water_system(1)
    W, tau, seed = 300, 0.005, 4321
    R0 = synth.initial_walkers(s, W, seed=8)
    e_cut = 0.2 * np.sqrt(s.n_elec / tau)
    # one DMC step through the handle-based entry point
    a = Q.QMC(s, seed=seed, cap_factor=4)
    a.set_walkers(R0)
    e_old = a.evaluate()["eloc"]
    e_trial = float(np.median(e_old))
    out = a.dmc(1, tau, e_trial)
    R1, _ = a.get_walkers()
    # the same sweep (same counter-based stream), then E_new from scratch
    b = Q.QMC(s, seed=seed, cap_factor=4)
    b.set_walkers(R0)
    b.vmc(1, tau)
    Rs, _ = b.get_walkers()
    e_new = b.evaluate()["eloc"]
    dev = torch.device("cuda", torch.cuda.current_device())
    eo = torch.tensor(e_old, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    p_full = None
    for call, en_host in enumerate((e_new, e_new)):
        en = torch.tensor(en_host, dtype=torch.float64, device=dev)
        parent = torch.full((4 * W,), -1, dtype=torch.int32, device=dev)
        stats = torch.zeros(5, dtype=torch.float64, device=dev)
        Q.qmc_branch_noalloc(eo, en, tau, e_trial, e_cut, seed, 0, parent, stats, stream)
        torch.cuda.synchronize()
        st = stats.cpu().numpy()
        Wn = int(st[2])
        assert st[3] == 0.0
        assert Wn == int(out["pop"][0]) == R1.shape[0], (call, Wn, out["pop"][0])
        p = parent.cpu().numpy()
        assert np.all(p[Wn:] == -1)
        p = p[:Wn]
        assert np.all(np.diff(p) >= 0) and p.min() >= 0 and p.max() < W
        assert np.max(np.abs(Rs[p] - R1)) < 1e-10
        assert abs(st[1] / st[0] - out["e_step"][0]) <= 1e-10 * max(1.0, abs(out["e_step"][0]))
        p_full = p
    # a smaller call after the larger ones: the first W2 walkers draw the same
    # uniforms (stream slot = walker index), so their copies are the larger
    # call's copies of those walkers; nothing the earlier calls left in the
    # scratch may leak into it
    W2 = 200
    parent = torch.full((4 * W,), -1, dtype=torch.int32, device=dev)
    stats = torch.zeros(5, dtype=torch.float64, device=dev)
    Q.qmc_branch_noalloc(eo[:W2].contiguous(), torch.tensor(e_new[:W2], dtype=torch.float64, device=dev),
                         tau, e_trial, e_cut, seed, 0, parent, stats, stream)
    torch.cuda.synchronize()
    st = stats.cpu().numpy()
    expect = p_full[p_full < W2]
    assert st[3] == 0.0 and int(st[2]) == expect.shape[0]
    p = parent.cpu().numpy()
    assert np.array_equal(p[:expect.shape[0]], expect) and np.all(p[expect.shape[0]:] == -1)
    # capacity below the new population: overflow flagged, parent untouched
    Wn = int(out["pop"][0])
    parent = torch.full((Wn - 1,), -1, dtype=torch.int32, device=dev)
    stats = torch.zeros(5, dtype=torch.float64, device=dev)
    Q.qmc_branch_noalloc(eo, torch.tensor(e_new, dtype=torch.float64, device=dev), tau, e_trial, e_cut, seed, 0,
                         parent, stats, stream)
    torch.cuda.synchronize()
    assert stats.cpu().numpy()[3] == 1.0
    assert np.all(parent.cpu().numpy() == -1)
    a.close()
    b.close()


def test_branch_noalloc_rejects_mismatched_buffers(Q):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    e = torch.zeros(16, dtype=torch.float64, device=dev)
    parent = torch.zeros(64, dtype=torch.int32, device=dev)
    stats = torch.zeros(5, dtype=torch.float64, device=dev)
    for bad in ((e, e[:8], parent, stats), (e, e.float(), parent, stats), (e, e, parent.long(), stats),
                (e, e, parent, stats[:4]), (e, e.cpu(), parent, stats)):
        with pytest.raises(ValueError):
            Q.qmc_branch_noalloc(bad[0], bad[1], 0.01, 0.0, 1.0, 1, 0, bad[2], bad[3])


def test_branch_noalloc_rejects_too_many_walkers(Q):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    W = 65536 + 1
    e = torch.zeros(W, dtype=torch.float64, device=dev)
    parent = torch.zeros(W, dtype=torch.int32, device=dev)
    stats = torch.zeros(5, dtype=torch.float64, device=dev)
    with pytest.raises(Q.QmcError) as ex:
        Q.qmc_branch_noalloc(e, e, 0.01, 0.0, 1.0, 1, 0, parent, stats)
    assert ex.value.code == -9
