"""The benchmark's CPU baseline (cpu_baseline/: the library's binary64 closed-form solid
code compiled for the host) against the oracle, on the CPU: codes bit-exact, distances and
safeties within 1e-9 mm, sentinels exact, on the precision-form solids, random solids of
every primitive kind, and the grazing-ray families.  Because the loop is the same source
as the GPU's binary64 pass, this also checks that source's closed forms without a GPU."""
import pytest

import cpu_baseline
import oracle
import workloads as W
from tests.helpers import compare

NAMED = {"box": W.BOX_M1, "trd": W.TRD_M3, "tube": W.TUBE_M2, "cone": W.CONE_M2, "polycone": W.polycone_m3()}
TABLE = W.solid_table(24, seed=11)


def _both(spec, tr):
    got = cpu_baseline.Solid(spec).query(**tr, threads=4)
    return got, oracle.Solid.from_spec(spec).query(**tr)


@pytest.mark.parametrize("name", list(NAMED))
def test_cpu_baseline_named(name):
    tr = W.tracks_for_solid(NAMED[name], 100_003, seed=500 + len(name))
    compare(*_both(NAMED[name], tr), "fp64", name)


@pytest.mark.parametrize("i", range(len(TABLE)))
def test_cpu_baseline_random_solids(i):
    tr = W.tracks_for_solid(TABLE[i], 20011, seed=600 + i)
    compare(*_both(TABLE[i], tr), "fp64", f"{TABLE[i]['kind']}#{i}")


@pytest.mark.parametrize("fam", W.GRAZING_FAMILIES)
def test_cpu_baseline_grazing(fam):
    spec, tr, _ = W.grazing_tracks(fam, 4000, 700 + W.GRAZING_FAMILIES.index(fam))
    compare(*_both(spec, tr), "fp64", fam)


@pytest.mark.parametrize("i", range(len(W.degenerate_table())))
def test_cpu_baseline_degenerate(i):
    spec = W.degenerate_table()[i]
    tr = W.tracks_for_solid(spec, 20011, seed=800 + i)
    compare(*_both(spec, tr), "fp64", f"degenerate {spec['kind']}#{i}")
