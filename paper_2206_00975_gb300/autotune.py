"""Autotuner of the batched launch geometry (ns_batched_tuning).

The batched solver (ns_solve_batched) has three launch knobs that do not
change its arithmetic: the panel width (columns of one problem per sketch work
item) and the persistent CTAs per SM of its sketch and dense kernels.  The best
setting depends on the GPU and on the batch's shapes, so it is measured: a
coordinate search over candidate values, each timed with CUDA events on a
sample of the batch, and the winner is cached in a JSON file under a key made
of (architecture, m' = 2^ceil(log2 m) of the largest problem, column panel =
the largest n rounded up to a power of two, dtype).  Later batches with the same
key reuse the cached setting without timing anything.

The tuner only marshals arguments and times library calls; every step of the
solve runs in the library's kernels.
"""
import json
import os

from . import api

DEFAULT = {"panel": 1, "sketch_ctas_per_sm": 0, "dense_ctas_per_sm": 0}
CANDIDATES = {"panel": [1, 2, 4], "sketch_ctas_per_sm": [0, 4, 2], "dense_ctas_per_sm": [0, 2, 1]}


def default_cache_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "batched_tuning.json")


def _pow2_ceil(x):
    x = max(int(x), 1)
    return 1 << (x - 1).bit_length()


def key_for(shapes, dtype, arch):
    """Cache key of a batch: shapes is a list of (m, n); dtype "f64" or "f32";
    arch e.g. "sm_103"."""
    mmax = max(m for m, _ in shapes)
    nmax = max(n for _, n in shapes)
    return "%s|mp=%d|npanel=%d|%s" % (arch, _pow2_ceil(mmax), _pow2_ceil(nmax), dtype)


def load_cache(path=None):
    path = path or default_cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=None):
    path = path or default_cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def coordinate_search(measure, candidates=None, start=None):
    """Tune one knob at a time (in the order of `candidates`), keeping the best
    value of each before moving to the next.  measure(setting) -> seconds.
    Returns (best setting, best time, list of (setting, time) tried)."""
    candidates = candidates or CANDIDATES
    best = dict(start or DEFAULT)
    best_t = measure(dict(best))
    tried = [(dict(best), best_t)]
    for knob, values in candidates.items():
        for v in values:
            if v == best[knob]:
                continue
            trial = dict(best)
            trial[knob] = v
            t = measure(trial)
            tried.append((dict(trial), t))
            if t < best_t:
                best, best_t = trial, t
    return best, best_t, tried


def _arch(torch):
    major, minor = torch.cuda.get_device_capability()
    return "sm_%d%d" % (major, minor)


def _dtype_name(problems):
    import torch
    return "f32" if any(p["A"].dtype == torch.float32 for p in problems) else "f64"


def tune_batched(problems, cache_path=None, sample=512, reps=2, stream=None):
    """Times the candidate settings on (up to) `sample` problems of the batch,
    caches and returns the best setting for the batch's key."""
    import torch
    sub = problems[:sample]
    ws = [None]

    def measure(setting):
        outs, st, keep = api.ns_solve_batched(sub, stream=stream, ws=ws[0], tuning=setting)
        ws[0] = keep[2]
        best = float("inf")
        for _ in range(reps):
            s = stream or torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            api.ns_solve_batched(sub, stream=stream, ws=ws[0], tuning=setting)
            e1.record(s)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return best

    best, best_t, tried = coordinate_search(measure)
    key = key_for([tuple(p["A"].shape) for p in problems], _dtype_name(problems), _arch(torch))
    cache = load_cache(cache_path)
    cache[key] = {"setting": best, "seconds_on_sample": best_t, "sample": len(sub),
                  "tried": [[s, t] for s, t in tried]}
    save_cache(cache, cache_path)
    return best


def lookup(problems, cache_path=None):
    """The cached setting for the batch's key, or None."""
    import torch
    key = key_for([tuple(p["A"].shape) for p in problems], _dtype_name(problems), _arch(torch))
    entry = load_cache(cache_path).get(key)
    return dict(entry["setting"]) if entry else None


def solve_batched_tuned(problems, cache_path=None, stream=None, ws=None):
    """ns_solve_batched with the cached setting for the batch's key, tuning
    (and caching) it first if there is none."""
    setting = lookup(problems, cache_path)
    if setting is None:
        setting = tune_batched(problems, cache_path=cache_path, stream=stream)
    return api.ns_solve_batched(problems, stream=stream, ws=ws, tuning=setting), setting
