"""Autotuner for the block-inversion kernel: picks the panel width and the
number of CTAs of the persistent factorization per species count S and
precision, by timing the library's own factorization phase (CUDA events
around it, xk_profile) on a short slice of the column.

Results are cached per (GPU name, S, precision) in a JSON file beside the
built library, and applied through xk_config.panel_width / factor_ctas.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import build as _build

CANDIDATES = {
    "fp64": [(8, 76), (8, 152), (16, 152), (4, 152)],
    "mixed": [(16, 76), (16, 152), (32, 38), (32, 76), (32, 152)],
}
CACHE = os.path.join(_build.BUILD, "autotune.json")


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(0)


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _key(S, precision):
    return f"{_gpu_name()}|S={S}|{precision}"


def measure(prob, precision, nb, ctas, layers=6, reps=2):
    """Factorization time per layer (ms) for one configuration."""
    import torch
    from . import xk
    sub = prob.replace(P_bar=prob.P_bar[:layers].copy(), T=prob.T[:layers].copy(),
                       Kzz=prob.Kzz[:layers].copy(), f0=prob.f0[:layers].copy())
    col = xk.Column(sub, precision, panel_width=nb, factor_ctas=ctas)
    col.set_mixing_ratios(sub.f0)
    n = col.get_state(device=True)
    col.step_delta(n, 1e-2)                   # warm-up (first launch, attribute set-up)
    col.profile(True)
    for _ in range(reps):
        col.step_delta(n, 1e-2)
    ms, calls = col.profile_read()["factor"]
    col.close()
    torch.cuda.synchronize()
    return ms / reps / layers


def tune(prob, precision, layers=6, verbose=False):
    """Time every candidate, cache and return (nb, ctas, table)."""
    table = []
    for nb, ctas in CANDIDATES[precision]:
        try:
            t = measure(prob, precision, nb, ctas, layers)
        except Exception as e:          # a candidate the library rejects (shared memory, size)
            if verbose:
                print(f"  nb={nb} ctas={ctas}: {e}")
            continue
        table.append((t, nb, ctas))
        if verbose:
            print(f"  {precision} S={prob.S} nb={nb:3d} ctas={ctas:4d}: {t:.3f} ms/layer", flush=True)
    if not table:
        raise RuntimeError("no factorization configuration ran")
    t, nb, ctas = min(table)
    data = _load()
    data[_key(prob.S, precision)] = {"panel_width": nb, "factor_ctas": ctas, "ms_per_layer": t,
                                     "table": [[x[1], x[2], x[0]] for x in table]}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    with open(CACHE, "w") as f:
        json.dump(data, f, indent=1)
    return nb, ctas, table


def tuned(S, precision):
    """Cached choice for (S, precision), or {} when not tuned yet."""
    e = _load().get(_key(S, precision))
    if not e:
        return {}
    return {"panel_width": int(e["panel_width"]), "factor_ctas": int(e["factor_ctas"])}


if __name__ == "__main__":
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2512_06729_gb300 import synth
    _build.build()
    for mk in (synth.full_column, synth.chons_column):
        p = mk()
        for prec in ("mixed", "fp64"):
            print(prec, p.S, tune(p, prec, verbose=True)[:2], flush=True)
    print(json.dumps(_load(), indent=1))
