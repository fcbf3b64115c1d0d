"""Autotuner: pick GEMM tile configurations and root-solver launch shapes by
timing them on the device (CUDA events), and remember the winners.

The paper leaves adaptive implementation selection to future work (Section 5,
item 1).  Here the candidates are the library's GEMM tile configurations
(mp_gemm_num_configs_P) and, for the batched Durand-Kerner solver, the block
size and blocks per SM of the persistent launch.  All candidates compute the
same bits; only their speed differs, so the choice is safe to cache.

Cache: a JSON file, $MPGPU_TUNE_CACHE or ~/.cache/mpgpu/tune.json, keyed by
device name, precision and a power-of-two size bucket.
"""

from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

_lock = threading.Lock()
_cache = None


def cache_path():
    return os.environ.get("MPGPU_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mpgpu", "tune.json"))


def _load():
    global _cache
    if _cache is None:
        try:
            with open(cache_path()) as f:
                _cache = json.load(f)
        except (OSError, ValueError):
            _cache = {}
    return _cache


def _save():
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(_cache, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass  # an unwritable cache only costs re-tuning


def _device():
    import torch

    return torch.cuda.get_device_name()


def _bucket(x):
    return 1 << max(0, int(math.ceil(math.log2(max(1, x)))))


def gemm_key(prec, m, n, k):
    return f"{_device()}|gemm|{prec}|{_bucket(m)}x{_bucket(n)}x{_bucket(k)}"


def best_gemm_config(prec, m, n, k):
    """Cached best configuration for this shape bucket, or -1 (built-in default)."""
    with _lock:
        return int(_load().get(gemm_key(prec, m, n, k), {}).get("config", -1))


def _time(fn, reps):
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_gemm(prec, m, n=None, k=None, reps=1, seed=0):
    """Time every tile configuration on seeded inputs of this shape; cache and
    return (best config, {config: ms})."""
    import torch

    from . import PRECS, empty, gemm, gemm_num_configs
    from . import inputs

    n = n or m
    k = k or m
    K = PRECS[prec][0]
    dt = np.float64 if PRECS[prec][1] == "float64" else np.float32
    A = torch.from_numpy(inputs.mp_uniform(seed, (m, k), K, dt, stream=inputs.STREAM_A)).cuda()
    B = torch.from_numpy(inputs.mp_uniform(seed, (k, n), K, dt, stream=inputs.STREAM_B)).cuda()
    C = empty(prec, m, n)
    times = {c: _time(lambda c=c: gemm(prec, A, B, out=C, config=c), reps)
             for c in range(gemm_num_configs(prec))}
    best = min(times, key=times.get)
    with _lock:
        _load()[gemm_key(prec, m, n, k)] = {"config": best, "ms": times}
        _save()
    return best, times


def roots_key(prec, npoly, max_degree):
    return f"{_device()}|roots|{prec}|{_bucket(npoly)}|{_bucket(max_degree)}"


def best_roots_shape(prec, npoly, max_degree):
    """Cached (threads, blocks_per_sm, engine) for this bucket, or (0, 0, 0) (built-in)."""
    with _lock:
        e = _load().get(roots_key(prec, npoly, max_degree))
    return (e["threads"], e["blocks_per_sm"], e.get("engine", 0)) if e else (0, 0, 0)


def tune_roots(prec, coef_off, coef, max_degree, sweeps=2, radius=1.1,
               candidates=((128, 0, 2), (256, 0, 1), (128, 0, 1), (64, 0, 1), (128, 2, 1))):
    """Time a few sweeps of the persistent batched solver for each (threads,
    blocks_per_sm, engine) candidate (engine 1 hybrid, 2 FP64 pipe; all give the
    same bits); cache and return the best and all timings."""
    from . import roots

    npoly = coef_off.numel() - 1
    times = {}
    for th, bps, eng in candidates:
        times[(th, bps, eng)] = _time(lambda th=th, bps=bps, eng=eng: roots(
            prec, coef_off, coef, max_degree, max_iter=sweeps, radius=radius, threads=th, blocks_per_sm=bps,
            sort=1, engine=eng), 1)
    best = min(times, key=times.get)
    with _lock:
        _load()[roots_key(prec, npoly, max_degree)] = {
            "threads": best[0], "blocks_per_sm": best[1], "engine": best[2],
            "ms": {f"{a}x{b}e{c}": v for (a, b, c), v in times.items()}}
        _save()
    return best, times
