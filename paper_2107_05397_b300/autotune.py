"""Autotuner driver: persistent cache of the library's tuned kernel settings.

The library times the candidates itself (`unifrac_autotune`, on the device,
CUDA events).  This module keys the winner by problem shape and keeps it in a
JSON file, so later contexts of similar shape start tuned without re-timing:

    key = variant, precision, largest-study bucket (power of 2), kept-branch
          bucket (power of 2), SM count

The dense / sparse splits are stored as fractions of the largest study so
that they carry over between sizes in the same bucket; the sparse kernels'
single-lane incidence bound and the weighted register flush length are
stored as they are.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

from . import binding as ub

# the package's cache of settings tuned on the GPUs this library is measured on
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


# options cached by value (name in the cache -> option id)
_PLAIN_OPTIONS = {"lane_pairs": ub.OPT_SPARSE_LANE_PAIRS,
                  "uw_lane_pairs": ub.OPT_UNWEIGHTED_SPARSE_LANE_PAIRS,
                  "flush": ub.OPT_WEIGHTED_FLUSH,
                  "rare_list": ub.OPT_RARE_LIST,
                  "uw_rare_list": ub.OPT_UNWEIGHTED_RARE_LIST}


def _bucket(x: float) -> int:
    return int(2 ** math.ceil(math.log2(max(1.0, float(x)))))


def _max_study(ctx: "ub.Context") -> int:
    so = ctx.study_offsets
    if so is None:
        return int(ctx.n_samples)
    return int(max(int(so[i + 1]) - int(so[i]) for i in range(len(so) - 1)))


def shape_key(ctx: "ub.Context", variant: int, precision: int) -> str:
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    kept = ctx.stat(ub.STAT_BRANCHES_KEPT)
    return (f"v{variant}-p{precision}-n{_bucket(_max_study(ctx))}-b{_bucket(kept)}-sm{sms}")


def tune(ctx: "ub.Context", variant: int, precision: int,
         cache_path: Optional[str] = None, repeats: int = 2) -> dict:
    """Apply cached settings for this shape, or time candidates and cache them."""
    import torch
    key = shape_key(ctx, variant, precision)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    n = _max_study(ctx)
    if key in cache:
        rec = cache[key]
        if "sparse_fraction" in rec:
            ctx.set_option(ub.OPT_SPARSE_THRESHOLD, max(2, int(round(rec["sparse_fraction"] * n))))
        if "uw_sparse_fraction" in rec:
            f = rec["uw_sparse_fraction"]
            ctx.set_option(ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD,
                           0 if f == 0 else max(2, int(round(f * n))))
        for name, opt in _PLAIN_OPTIONS.items():
            if name in rec:
                ctx.set_option(opt, int(rec[name]))
        return dict(rec, cached=True)
    nbytes = ctx.output_bytes(precision, ub.OUT_CONDENSED)
    out = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device="cuda")
    ub.unifrac_autotune(ctx.handle, variant, precision, out, repeats)
    rec = {}
    if variant == ub.WEIGHTED_NORMALIZED and precision == ub.MIXED:
        rec["sparse_fraction"] = ub.unifrac_get_option(ctx.handle, ub.OPT_SPARSE_THRESHOLD) / max(n, 1)
    if variant == ub.UNWEIGHTED and precision == ub.MIXED:
        rec["uw_sparse_fraction"] = ub.unifrac_get_option(ctx.handle, ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD) / max(n, 1)
    if precision == ub.MIXED:
        mine = (("lane_pairs", "flush", "rare_list") if variant == ub.WEIGHTED_NORMALIZED
                else ("uw_lane_pairs", "uw_rare_list"))
        for name in mine:
            rec[name] = ub.unifrac_get_option(ctx.handle, _PLAIN_OPTIONS[name])
    if cache_path:
        cache[key] = rec
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return dict(rec, cached=False)
