"""The parameter sweep's steady-state agreement rule (paper_1906_11027_gb300.sweep)
on a 40-domain draw of the sweep (seed 11027: sides 64..256, G in [-5.5, -4.3],
tau in {0.6, 0.8, 1.0}, R in [8, 0.35 L], stencil orders 4..10).

Both batched FP32 arms -- from the tanh start and from the learned warm start,
the network trained first on 40 other domains (seed 11028) -- are compared with
the plain FP64 method run one domain per launch.  Every domain's steady max|u|
must agree within 5% or fall in one of the rule's stated classes (both
diverged, both below FP32's velocity resolution, a different basin, a run
that passed the steady test early and agrees once continued to the other's
step count, or -- for the learned start -- a domain on which both tanh-started
runs diverged); none may be left unexplained.  Most domains agree outright.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_every_sweep_domain_agrees_or_is_classified(lbm):
    from paper_1906_11027_gb300 import inputs, sweep, warmstart

    doms = inputs.sweep_domains(40)
    tdoms = inputs.sweep_domains(40, seed=inputs.SWEEP_SEED + 1)
    tb = lbm.Batch(tdoms, precision=lbm.LBM_FP32_SHIFTED)
    _, tobs, _ = tb.run_to_steady(sweep.TOL, 200000, sweep.K)
    Xt, yt, _, _, _ = warmstart.dataset_from_batch(tb, tdoms, tobs)
    tb.close()
    net, _ = warmstart.train(Xt, yt, epochs=30)

    plain = sweep.batched(doms)
    warm = sweep.batched(doms, net)
    ref = sweep.one_per_launch(doms, keep_if=sweep.misses_5pct(plain, warm))
    for name, arm, tanh_arm in (("tanh", plain, None), ("warm", warm, plain)):
        cls = sweep.classify(doms, arm, ref, tanh_arm=tanh_arm)
        n = sweep.counts(cls)
        bad = [(i, doms[i], arm["obs"][i]["max_u"], ref["obs"][i]["max_u"], arm["steps"][i], ref["steps"][i])
               for i, c in enumerate(cls) if c == "unexplained"]
        assert not bad, (name, n, bad)
        compared = len(doms) - n["diverged_both"] - n["tanh_start_diverged"]
        assert n["within_5pct"] >= 0.8 * compared, (name, n)
    plain["batch"].close()
    warm["batch"].close()
