"""Shared helpers for the GPU parity tests: seeded tracks to the device, the
library's results back to numpy, and the comparison rules.

Comparison rules (the stated tolerances):
  * inside codes: bit-exact;
  * FP64 pass: |distance or safety - oracle| <= 1e-9 mm;
  * FP32 + refinement pass: relative 1e-5, absolute 1e-9 mm below 1e-4 mm;
  * the sentinels (-1 wrong side, +inf no entry) and zeros must match exactly.
"""
import numpy as np

QUERIES = ("inside", "dist_in", "dist_out", "safety_in", "safety_out")


def to_device(tracks, torch):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in tracks.items()}


def to_host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def compare(got, want, mode="fp64", label=""):
    """Assert parity; return per-query error statistics."""
    stats = {}
    if "inside" in got:
        gi, wi = got["inside"], want["inside"]
        bad = np.nonzero(gi != wi)[0]
        assert len(bad) == 0, (f"{label}: {len(bad)} inside-code mismatches, first {bad[:5]} "
                               f"got {gi[bad[:5]]} want {wi[bad[:5]]}")
    for k in QUERIES[1:]:
        if k not in got:
            continue
        g, w = got[k], want[k]
        special = ~np.isfinite(w) | (w == -1.0) | (w == 0.0)
        gs = ~np.isfinite(g) | (g == -1.0) | (g == 0.0)
        mism = np.nonzero(special & ~((g == w) | (np.isinf(g) & np.isinf(w))))[0]
        assert len(mism) == 0, f"{label} {k}: sentinel mismatch at {mism[:5]} got {g[mism[:5]]} want {w[mism[:5]]}"
        fin = ~special
        extra = np.nonzero(fin & gs)[0]
        assert len(extra) == 0, f"{label} {k}: sentinel where the oracle has a value at {extra[:5]} got {g[extra[:5]]} want {w[extra[:5]]}"
        err = np.abs(g[fin] - w[fin])
        if mode == "fp64":
            badv = np.nonzero(err > 1e-9)[0]
        else:
            tol = np.where(np.abs(w[fin]) < 1e-4, 1e-9, 1e-5 * np.abs(w[fin]))
            badv = np.nonzero(err > tol)[0]
        idx = np.nonzero(fin)[0]
        assert len(badv) == 0, (f"{label} {k}: {len(badv)} values out of tolerance, worst "
                                f"{err.max():.3e} at {idx[badv[:5]]} got {g[idx[badv[:5]]]} want {w[idx[badv[:5]]]}")
        rel = err / np.maximum(np.abs(w[fin]), 1e-300)
        stats[k] = {"max_abs": float(err.max()) if err.size else 0.0,
                    "max_rel": float(rel.max()) if rel.size else 0.0,
                    "p9999_rel": float(np.quantile(rel, 0.9999)) if rel.size else 0.0}
    return stats
