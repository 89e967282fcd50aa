"""Batched evaluation (many baskets, each against its own solid, persistent kernels per
solid family replayed from one CUDA graph), checked against the CPU oracle.

The full batched workload (4096 baskets of 16-4096 tracks over 64 solids of the
six types) is small enough for the oracle to check every track.  Also: results
of a basket are bit-identical alone and in the mix, across launch shapes and
after autotuning; empty baskets and one-track baskets.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.helpers import QUERIES, compare, to_device, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gv():
    import torch  # noqa: F401
    import paper_1512_06637_gb300 as gv
    from paper_1512_06637_gb300 import build
    build.build()
    return gv


@pytest.fixture(scope="module")
def work():
    return W.batched()


def oracle_all(work):
    n = len(work["tracks"]["x"])
    want = {k: np.empty(n, np.int8 if k == "inside" else np.float64) for k in QUERIES}
    by_solid = {}
    for b in range(len(work["n"])):
        by_solid.setdefault(int(work["solid"][b]), []).append(
            np.arange(work["offset"][b], work["offset"][b] + work["n"][b]))
    for sid, parts in by_solid.items():
        idx = np.concatenate(parts)
        sub = {k: v[idx] for k, v in work["tracks"].items()}
        r = oracle.Solid.from_spec(work["solids"][sid]).query(**sub)
        for k in QUERIES:
            want[k][idx] = r[k]
    return want


@pytest.fixture(scope="module")
def want(work):
    return oracle_all(work)


def make_batch(gv, work):
    solids = [gv.Solid.from_spec(s) for s in work["solids"]]
    return gv.Batch(solids, work["offset"], work["n"], work["solid"])


@pytest.mark.parametrize("precision", ["fp32_refine", "fp64"])
def test_batched_parity_full(gv, work, want, precision):
    import torch
    b = make_batch(gv, work)
    dev = to_device(work["tracks"], torch)
    n = dev["x"].numel()
    out = gv.alloc_results(n, "cuda")
    b.run(dev, out, precision=precision)
    b.run(dev, out, precision=precision)  # graph replay
    torch.cuda.synchronize()
    compare(to_host(out), want, "fp32" if precision == "fp32_refine" else "fp64", f"batched-{precision}")
    if precision == "fp32_refine":
        print("batched refined fraction", b.refined() / n)


def test_batched_alone_equals_mix_and_shapes(gv, work):
    """Per-track math does not depend on neighbours: a basket's results are the same
    bits alone (single-solid query), in the mix, and under every launch shape."""
    import torch
    b = make_batch(gv, work)
    dev = to_device(work["tracks"], torch)
    n = dev["x"].numel()
    ref = gv.alloc_results(n, "cuda")
    b.run(dev, ref)
    torch.cuda.synchronize()
    for threads, items, ctas in ((128, 1, 1), (512, 4, 0), (256, 2, 2)):
        b.set_config(threads, items, ctas)
        out = gv.alloc_results(n, "cuda")
        b.run(dev, out)
        torch.cuda.synchronize()
        for k in QUERIES:
            assert torch.equal(out[k], ref[k]), (threads, items, ctas, k)
    ws = gv.Workspace(5000)
    for bi in (0, 17, 4095):
        o, m, sid = int(work["offset"][bi]), int(work["n"][bi]), int(work["solid"][bi])
        sub = {k: v[o:o + m].contiguous() for k, v in dev.items()}
        alone = gv.query(gv.Solid.from_spec(work["solids"][sid]), sub, precision="fp32_refine", workspace=ws)
        torch.cuda.synchronize()
        for k in QUERIES:
            assert torch.equal(alone[k], ref[k][o:o + m]), (bi, k)


def test_batched_fp64_ordered_tiles_same_bits(gv, work):
    """The binary64 batched kernel evaluates each tile in work-class order: every basket's
    results are the same bits as the single-solid binary64 pass in index order, under several
    launch shapes (tiles of 128 to 2048 tracks)."""
    import torch
    b = make_batch(gv, work)
    dev = to_device(work["tracks"], torch)
    n = dev["x"].numel()
    outs = []
    for threads, items, ctas in ((128, 1, 1), (512, 4, 0), (256, 2, 2)):
        b.set_config(threads, items, ctas)
        out = gv.alloc_results(n, "cuda")
        b.run(dev, out, precision="fp64")
        torch.cuda.synchronize()
        outs.append(out)
    for bi in (0, 17, 1000, 4095):
        o, m, sid = int(work["offset"][bi]), int(work["n"][bi]), int(work["solid"][bi])
        sub = {k: v[o:o + m].contiguous() for k, v in dev.items()}
        alone = gv.query(gv.Solid.from_spec(work["solids"][sid]), sub, precision="fp64")
        torch.cuda.synchronize()
        for out in outs:
            for k in QUERIES:
                assert torch.equal(alone[k], out[k][o:o + m]), (bi, k)


def test_batched_autotune(gv, work, want):
    import torch
    b = make_batch(gv, work)
    dev = to_device(work["tracks"], torch)
    n = dev["x"].numel()
    out = gv.alloc_results(n, "cuda")
    best = b.autotune(dev, out)
    assert best["threads"] in (128, 256, 512) and best["items"] in (1, 2, 4)
    assert b.config() == best
    b.run(dev, out)
    torch.cuda.synchronize()
    compare(to_host(out), want, "fp32", "batched-autotuned")


def test_batched_empty_and_tiny_baskets(gv):
    import torch
    solids_spec = [W.BOX_M1, W.TUBE_M2, W.polycone_m3()]
    solids = [gv.Solid.from_spec(s) for s in solids_spec]
    sizes = [0, 1, 0, 3, 1000, 0, 1]
    sid = [0, 1, 2, 2, 1, 0, 0]
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    total = int(sum(sizes))
    parts = [W.tracks_for_solid(solids_spec[s], max(m, 1), seed=70 + i) for i, (m, s) in enumerate(zip(sizes, sid))]
    tr = {k: np.concatenate([p[k][:m] for p, m in zip(parts, sizes)]) for k in parts[0]}
    b = gv.Batch(solids, offs, sizes, sid)
    dev = to_device(tr, torch)
    out = gv.alloc_results(total, "cuda")
    b.run(dev, out)
    torch.cuda.synchronize()
    got = to_host(out)
    for i, (m, s) in enumerate(zip(sizes, sid)):
        if m == 0:
            continue
        o = int(offs[i])
        sub = {k: v[o:o + m] for k, v in tr.items()}
        w = oracle.Solid.from_spec(solids_spec[s]).query(**sub)
        compare({k: v[o:o + m] for k, v in got.items()}, w, "fp32", f"basket{i}")


def test_batched_rejects_bad_tables(gv):
    import ctypes
    from paper_1512_06637_gb300 import _abi
    s = gv.Solid.from_spec(W.BOX_M1)
    with pytest.raises(gv.GVError):
        gv.Batch([s], [0], [10], [1])  # unknown solid
    with pytest.raises(gv.GVError):
        gv.Batch([s], [-1], [10], [0])  # negative offset
    h = ctypes.c_void_p()
    assert _abi.lib().gv_batch_create(None, 0, None, 0, ctypes.byref(h)) == 1
