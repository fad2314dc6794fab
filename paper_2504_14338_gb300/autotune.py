"""Autotuner for the launch schedules of the learn and reduce steps.

Two knobs decide how the work is laid out on the GPU without changing a single bit of the
results (both choices are exercised by the GPU tests):

* how many operator rows each CTA of a rollout cluster owns (1, 2, 4 or 8 for r <= 32, 3 to 8 for
  r above 32, so ceil(r / rows) CTAs per candidate): large clusters shorten each candidate's
  chain of evaluations, small ones leave more of the GPU's issue slots to the other candidates;
* the Householder tridiagonalisation as one cooperative launch (a grid barrier per column) or
  as three launches per column.

`tune_learn` and `tune_reduce` time each setting on the caller's own inputs with the CUDA
events the library records (the rollout stage of dopinf_learn) or around the call, keep the
fastest, set it process-wide and return the table.  Results are cached per device and shape
key, so a workload is tuned once per process.
"""
import torch

from . import dopinf as dp

_cache = {}


def pick_fastest(times):
    """The setting with the smallest time (the first one on ties): the selection rule."""
    best = None
    for setting, t in times.items():
        if best is None or t < times[best]:
            best = setting
    return best


def _key(kind, *parts):
    return (kind, torch.cuda.get_device_name(), *parts)


def tune_learn(Qhat, r_list, beta1, beta2, n_steps, mode=dp.DISCRETE, dt=1.0, rows=(1, 2, 4, 8),
               rows_large=(3, 4, 5, 6, 8), reps=3, ws=None, timer=None):
    """Time the rollouts of this grid search for each launch shape; set and return the best.

    Two knobs, tuned one after the other (the other one held at its current value): operator
    rows per CTA of the rollouts of r <= 32 (`rows`) if the list has such an r, and of the
    rollouts of r > 32 (`rows_large`) if it has such an r.  timer(knob, setting) ->
    milliseconds replaces the measurement (host-logic tests).  The result names the first
    knob tuned ("knob", "best", "rollout_ms") and lists all of them under "knobs"."""
    knobs = []
    if min(int(r) for r in r_list) <= 32:
        knobs.append(("rollout rows per CTA", dp.dopinf_tune_rollout_rows, rows))
    if max(int(r) for r in r_list) > 32:
        knobs.append(("rollout rows per CTA (r > 32)", dp.dopinf_tune_rollout_rows_large, rows_large))
    key = _key("learn", tuple(r_list), len(beta1), len(beta2), int(n_steps), int(mode), int(Qhat.shape[1]))
    if timer is None and key in _cache:
        for (name, setter, _), k in zip(knobs, _cache[key]["knobs"]):
            setter(k["best"])
        return _cache[key]
    results = []
    for name, setter, settings in knobs:
        prev = setter(0)
        times = {}
        try:
            for c in settings:
                if timer is not None:
                    times[c] = float(timer(name, c))
                    continue
                setter(c)
                best_ms = None
                for _ in range(reps + 1):  # the first run warms up
                    res = dp.dopinf_learn(Qhat, r_list, beta1, beta2, n_steps, mode=mode, dt=dt, ws=ws)
                    ms = res["stage_ms"]["rollouts"]
                    best_ms = ms if best_ms is None else min(best_ms, ms)
                times[c] = best_ms
        finally:
            setter(prev)
        best = pick_fastest(times)
        setter(best)
        results.append({"knob": name, "best": best, "rollout_ms": times})
    out = dict(results[0])
    out["knobs"] = results
    if timer is None:
        _cache[key] = out
    return out


def tune_reduce(D, r_cap, r_fixed=None, reps=3, ws=None, timer=None):
    """Time dopinf_reduce with the cooperative tridiagonalisation on and off; set and return the best."""
    k = int(D.shape[0])
    key = _key("reduce", k, int(r_cap))
    if timer is None and key in _cache:
        dp.dopinf_tune_reduce_coop(_cache[key]["best"])
        return _cache[key]
    prev = dp.dopinf_tune_reduce_coop(-1)
    times = {}
    stream = torch.cuda.current_stream() if timer is None else None
    try:
        for on in (1, 0):
            if timer is not None:
                times[on] = float(timer(on))
                continue
            dp.dopinf_tune_reduce_coop(on)
            best_ms = None
            for _ in range(reps + 1):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                dp.dopinf_reduce(D, r_cap=r_cap, r_fixed=r_cap if r_fixed is None else r_fixed, ws=ws)
                b.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                best_ms = ms if best_ms is None else min(best_ms, ms)
            times[on] = best_ms
    finally:
        dp.dopinf_tune_reduce_coop(prev)
    best = pick_fastest(times)
    dp.dopinf_tune_reduce_coop(best)
    out = {"knob": "cooperative tridiagonalisation", "best": best, "reduce_ms": times}
    if timer is None:
        _cache[key] = out
    return out
