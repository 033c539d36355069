"""The parameter sweep's arms and the rule that compares their steady states.

Arms (each runs every domain of the draw to steady state under the same rule,
|max|u|(t) - max|u|(t - K)| / K < tol checked every K = 100 steps, FP32 storage
adding the floor 1e-6 max|u| / K for its round-off):
- batched: every domain in one persistent-kernel CUDA graph with FP32
  deviation storage, from the tanh start or from the learned warm start.  The
  tanh start is the learned start's fallback: a domain that diverges from the
  learned start runs again from the tanh start, its steps and time counted in
  the learned-start arm.  A domain whose steady max|u| is below FP32's
  velocity resolution (fp64_below) is continued in FP64 from its FP32 state
  (the precision policy of the batched sweep);
- one_per_launch: the plain method, one FP64 domain per launch, tanh start.

Agreement rule: a domain's steady max|u| in a batched arm agrees with the FP64
arm when the relative difference is at most 5%.  A domain that misses falls in
exactly one of these classes, checked in this order:
- diverged_both: both arms diverged (BGK is unstable for some strong-G,
  small-tau pairs; such a domain retires with max|u| = inf in both);
- below_resolution: both currents are below fp64_below, where FP32 storage
  cannot resolve a relative difference;
- other_basin: one current is below fp64_below and the other is not: near the
  critical coupling the droplet dissolves in one run and survives in the other;
- stopped_early: the two runs passed the steady test at different step counts,
  and the one that stopped first, continued in FP64 from its final state to
  the other's step count, agrees within 5%.  The steady test compares max|u|
  over one window, so it can pass at a turning point of a slowly evolving
  current; continuing the run shows whether the two states differ only in how
  far they had evolved;
- tanh_start_diverged: for the learned-start arm only, both tanh-started runs
  (FP64 and batched FP32) diverged and the learned start reached a steady
  state.  At strong G and small tau the tanh start's transient, from densities
  far from coexistence, drives BGK unstable; the learned start begins near the
  steady profile and avoids it;
- unexplained: anything else (also a domain that diverged in one arm only
  for any other reason).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import lbm

K = 100
TOL = 1e-10
FP64_BELOW = 1e-6
CLASSES = ("within_5pct", "diverged_both", "below_resolution", "other_basin", "stopped_early",
           "tanh_start_diverged", "unexplained")


def _sync():
    import torch
    torch.cuda.synchronize()


def batched(doms, net=None, max_steps=200000, fp64_below=FP64_BELOW):
    """The batched FP32 arm.  Returns a dict with wall time, per-domain steps and
    observables, and the live Batch (for the final states; close it when done)."""
    from . import warmstart
    t0 = time.perf_counter()
    b = lbm.Batch(doms, precision=lbm.LBM_FP32_SHIFTED)
    fallbacks = warmstart.batch_warm_init(b, doms, net) if net is not None else None
    t_init = time.perf_counter() - t0
    steps, obs, ok = b.run_to_steady(TOL, max_steps, K)
    steps, obs = list(steps), list(obs)
    evolved = list(steps)  # steps of the run that produced each final state
    states64 = {}  # final states kept outside the batch
    restarted = []
    if net is not None:
        # the tanh start is the learned start's fallback: a domain that diverged
        # from the learned start runs again from the tanh start (its steps add up)
        restarted = [i for i, o in enumerate(obs) if not np.isfinite(o["max_u"])]
        if restarted:
            br = lbm.Batch([doms[i] for i in restarted], precision=lbm.LBM_FP32_SHIFTED)
            sr, orr, okr = br.run_to_steady(TOL, max_steps, K)
            ok = ok and okr
            for j, i in enumerate(restarted):
                steps[i] += sr[j]
                evolved[i] = sr[j]
                obs[i] = orr[j]
                states64[i] = br.get_f(j)
            br.close()
    _sync()
    t_fp32 = time.perf_counter() - t0
    tiny = [i for i, o in enumerate(obs) if np.isfinite(o["max_u"]) and o["max_u"] < fp64_below]
    if tiny:
        b64 = lbm.Batch([doms[i] for i in tiny], precision=lbm.LBM_FP64)
        for j, i in enumerate(tiny):
            b64.set_f(j, states64[i] if i in states64 else b.get_f(i))
        s64, o64, _ = b64.run_to_steady(TOL, max_steps, K)
        for j, i in enumerate(tiny):
            steps[i] += s64[j]
            evolved[i] += s64[j]
            obs[i] = o64[j]
            states64[i] = b64.get_f(j)
        b64.close()
    _sync()
    return dict(t=time.perf_counter() - t0, t_init=t_init, t_fp32=t_fp32, steps=list(steps), evolved=evolved,
                obs=list(obs), ok=ok, tiny=len(tiny), fallbacks=fallbacks, restarted=len(restarted), schedule=b.schedule_report(),
                batch=b, states64=states64)


def batched_state(arm, i):
    """Final populations (double, [9][1][ny][nx]) of domain i of a batched arm."""
    return arm["states64"][i] if i in arm["states64"] else arm["batch"].get_f(i)


def one_per_launch(doms, max_steps=200000, keep_if=None):
    """The plain FP64 method, one domain per launch, tanh start.  The final state
    of domain i is kept (for classify) when keep_if(i, max_u) is true."""
    t0 = time.perf_counter()
    steps, obs, states = [], [], []
    for d in doms:
        dom = lbm.Domain(d["nx"], d["ny"], G=d["G"], tau=d["tau"], stencil=d["stencil"], precision=lbm.LBM_FP64)
        dom.init_droplet(d["rho_l"], d["rho_g"], d["R"], d["width"])
        try:
            s, _ = dom.run_to_steady(TOL, max_steps, K)
            o = dom.observables()
            f = dom.get_f() if keep_if is not None and keep_if(len(steps), o["max_u"]) else None
        except lbm.LbmError as e:  # the BGK model diverges for some (G, tau) pairs
            if e.code != lbm.LBM_ENONFINITE:
                raise
            s, o, f = max_steps, {"max_u": float("inf")}, None
        steps.append(s)
        obs.append(o)
        states.append(f)
        dom.close()
    _sync()
    return dict(t=time.perf_counter() - t0, steps=steps, obs=obs, states=states)


def _continued_max_u(d, f, nsteps):
    dom = lbm.Domain(d["nx"], d["ny"], G=d["G"], tau=d["tau"], stencil=d["stencil"], precision=lbm.LBM_FP64)
    dom.set_f(f)
    dom.step(int(nsteps))
    u = dom.observables()["max_u"]
    dom.close()
    return u


def classify(doms, arm, ref, fp64_below=FP64_BELOW, tanh_arm=None):
    """The class of every domain (see the module docstring) of a batched arm
    against the FP64 one-per-launch arm (its states kept where they may be
    needed: misses_5pct gives the keep_if for that).  For the learned-start
    arm, tanh_arm is the batched arm from the tanh start."""
    out = []
    for i, d in enumerate(doms):
        ua, ub = arm["obs"][i]["max_u"], ref["obs"][i]["max_u"]
        fa, fb = math.isfinite(ua), math.isfinite(ub)
        if not fa and not fb:
            out.append("diverged_both")
        elif fa and not fb and tanh_arm is not None and not math.isfinite(tanh_arm["obs"][i]["max_u"]):
            out.append("tanh_start_diverged")
        elif fa != fb:
            out.append("unexplained")
        elif abs(ua / ub - 1.0) <= 0.05:
            out.append("within_5pct")
        elif max(ua, ub) < fp64_below:
            out.append("below_resolution")
        elif min(ua, ub) < fp64_below:
            out.append("other_basin")
        else:
            sa, sb = arm.get("evolved", arm["steps"])[i], ref["steps"][i]
            if sa < sb:
                u = _continued_max_u(d, batched_state(arm, i), sb - sa)
                ok = abs(u / ub - 1.0) <= 0.05
            elif sb < sa and ref["states"][i] is not None:
                u = _continued_max_u(d, ref["states"][i], sa - sb)
                ok = abs(ua / u - 1.0) <= 0.05
            else:
                ok = False
            out.append("stopped_early" if ok else "unexplained")
    return out


def misses_5pct(*arms):
    """keep_if for one_per_launch: domain i misses 5% against one of the arms."""
    def keep(i, u):
        for a in arms:
            ua = a["obs"][i]["max_u"]
            if not (math.isfinite(ua) and math.isfinite(u)) or abs(ua / u - 1.0) > 0.05:
                return True
        return False
    return keep


def counts(classes):
    return {c: sum(1 for k in classes if k == c) for c in CLASSES}
