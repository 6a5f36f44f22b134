"""Persistent cache for the query kernel's autotuned ring geometry.

The library's autotuners (kerdock_plan_tune, kerdock_batch_tune) time every
candidate ring geometry on the GPU; this module remembers the winner per
device and problem shape in a JSON file so later processes skip the search.
The cache file is $KERDOCK_TUNING_CACHE, else ~/.cache/kerdock_tuning.json.
"""
import json
import os

from . import kerdock as K


def cache_path():
    return os.environ.get("KERDOCK_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "kerdock_tuning.json"))


def _load():
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(table):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _device_name():
    import torch
    return torch.cuda.get_device_name()


def plan_key(plan, q):
    i = plan.info
    qb = 1 << max(0, int(q) - 1).bit_length()  # power-of-two bucket of the batch size
    return f"{_device_name()}|plan|m{i['m']}|n{i['n']}|t{i['dtype']}|J{i['J']}|K{i['K']}|S{i['S']}|q{qb}"


def autotune_plan(plan, X, eps, seed, reps=3, use_cache=True):
    """Pick the ring geometry for plan.apply(X, ...), from the cache or by timing."""
    key = plan_key(plan, X.shape[0])
    table = _load() if use_cache else {}
    if key in table:
        rk, cr = table[key]["ring_kb"], table[key]["crows"]
        K.kerdock_plan_set_tuning(plan.handle, rk, cr)
        return rk, cr, table[key].get("ms")
    idx, val, cnt = plan.alloc_outputs(X.shape[0])
    ws = plan.workspace(X.shape[0])
    wsp, wsb = (ws.data_ptr(), ws.numel()) if ws is not None else (None, 0)
    plan._sync_stream()
    rk, cr, ms = K.kerdock_plan_tune(plan.handle, X.data_ptr(), X.shape[0], X.stride(0), float(eps),
                                     int(seed), idx.data_ptr(), val.data_ptr(), cnt.data_ptr(),
                                     wsp, wsb, reps)
    if use_cache:
        table = _load()
        table[key] = {"ring_kb": rk, "crows": cr, "ms": ms}
        _store(table)
    return rk, cr, ms


def batch_key(batch):
    shapes = sorted({(sp["plan"].info["n"], sp["plan"].info["dtype"]) for sp in batch.specs})
    return f"{_device_name()}|batch|{len(batch.specs)}|" + ",".join(f"{n}:{t}" for n, t in shapes)


def autotune_batch(batch, reps=3, use_cache=True):
    key = batch_key(batch)
    table = _load() if use_cache else {}
    if key in table:
        batch.set_tuning(table[key]["ring_kb"], table[key]["crows"])
        return table[key]["ring_kb"], table[key]["crows"], table[key].get("ms")
    rk, cr, ms = batch.tune(reps)
    if use_cache:
        table = _load()
        table[key] = {"ring_kb": rk, "crows": cr, "ms": ms}
        _store(table)
    return rk, cr, ms
