"""The step-reduction hook of sharded DMC on one GPU, through the C ABI.

qmc_set_step_reduce hands every DMC step's sums to a callback that must
return their sum over ranks.  On one GPU: the identity (one rank) must
reproduce the plain run exactly; doubling every sum (two identical ranks)
must leave every ratio -- step energy, trial energy, population feedback,
force estimator -- unchanged (a factor 2 is exact in floating point); a
failing callback fails the step; and a one-rank gloo group through
shard.StepReducer is the identity.
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


def run(Q, reduce_fn=None, fixed=False, ref=None):
    s = synth.water_system(1)
    g = Q.QMC(s, seed=55, cap_factor=4, fixed_population=fixed)
    g.set_walkers(synth.initial_walkers(s, 48, seed=9))
    if reduce_fn is not None:
        Q.qmc_set_step_reduce(g.h, reduce_fn)
    if ref is not None:
        Q.qmc_set_population_reference(g.h, ref)
    out = g.dmc(6, 0.005, -70.0, forces_every=2)
    F, _ = g.force_estimate(Q.QMC_EST_DMC)
    g.close()
    return out, F


def _scale(f):
    def fn(buf, n, ctx):
        for i in range(n):
            buf[i] *= f
        return 0
    return fn


@pytest.mark.parametrize("fixed", [False, True])
def test_identity_and_two_identical_ranks_reproduce_the_plain_run(Q, fixed):
    base, F0 = run(Q, fixed=fixed)
    ident = Q.REDUCE_FN(_scale(1.0))
    out1, F1 = run(Q, ident, fixed=fixed)
    for k in ("e_step", "pop", "e_trial"):
        assert np.array_equal(out1[k], base[k]), k
    assert np.array_equal(F1, F0)
    # two identical ranks: the sums double, the reference population too
    double = Q.REDUCE_FN(_scale(2.0))
    out2, F2 = run(Q, double, fixed=fixed)
    for k in ("e_step", "pop", "e_trial"):
        assert np.array_equal(out2[k], base[k]), k
    assert np.array_equal(F2, F0)


def test_reference_population_and_failing_callback(Q):
    base, _ = run(Q)
    # a reference population equal to the initial one changes nothing
    same, _ = run(Q, ref=48.0)
    assert np.array_equal(same["e_trial"], base["e_trial"])
    # a different reference shifts the feedback term by ln(48 / ref) / (10 tau)
    other, _ = run(Q, ref=96.0)
    assert np.allclose(other["e_trial"][0] - base["e_trial"][0], np.log(2.0) / 0.05, rtol=1e-12)
    bad = Q.REDUCE_FN(lambda buf, n, ctx: 1)
    s = synth.water_system(1)
    g = Q.QMC(s, seed=55, cap_factor=4)
    g.set_walkers(synth.initial_walkers(s, 48, seed=9))
    Q.qmc_set_step_reduce(g.h, bad)
    with pytest.raises(Q.QmcError) as ex:
        g.dmc(1, 0.005, -70.0)
    assert ex.value.code == -7
    Q.qmc_set_step_reduce(g.h, None)
    g.close()


def test_one_rank_gloo_group_is_the_identity(Q, tmp_path):
    import torch.distributed as dist
    from paper_2504_07948_gb300 import shard
    dist.init_process_group("gloo", init_method=f"file://{tmp_path}/store", rank=0, world_size=1)
    try:
        base, F0 = run(Q)
        s = synth.water_system(1)
        g = Q.QMC(s, seed=55, cap_factor=4)
        g.set_walkers(synth.initial_walkers(s, 48, seed=9))
        red = shard.StepReducer()
        shard.attach(g, red)
        out = g.dmc(6, 0.005, -70.0, forces_every=2)
        F, _ = g.force_estimate(Q.QMC_EST_DMC)
        assert red.calls == 6
        assert np.array_equal(out["e_step"], base["e_step"]) and np.array_equal(F, F0)
        assert shard.rebalance(g) == []
        shard.detach(g)
        g.close()
    finally:
        dist.destroy_process_group()
