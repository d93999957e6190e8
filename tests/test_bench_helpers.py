"""CPU checks of the benchmark's measurement helpers: the cell census that the
roofline's algorithmic work is counted from, against a brute-force count."""
import itertools
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench


def _brute_census(gamma, spacing, dta):
    """For every evaluated voxel v and every grid cube (lower corner v + c at
    0 .. n - 2 on each axis, so the whole cube lies inside the grid): count it
    when its box distance / dta is below gamma(v), split into the cubes whose
    box contains v (distance 0) and the others; each evaluated voxel adds one
    to the first count (its final stop test)."""
    nd = gamma.ndim
    shape = gamma.shape                                  # (z, y, x) or (y, x)
    hn = np.array(spacing[::-1], dtype=np.float64) / dta  # x, y[, z]
    dims = shape[::-1]
    shell = tail = 0
    for idx in itertools.product(*[range(n) for n in shape]):
        g = gamma[idx]
        if not np.isfinite(g):
            continue
        v = idx[::-1]                                    # x, y[, z]
        shell += 1
        lim = [int(math.ceil(g / h)) + 1 for h in hn]
        for c in itertools.product(*[range(-l - 1, l + 1) for l in lim]):
            if any(not (0 <= v[a] + c[a] <= dims[a] - 2) for a in range(nd)):
                continue
            gap = [max(c[a], -c[a] - 1, 0) * hn[a] for a in range(nd)]
            key = math.sqrt(sum(x * x for x in gap))
            if key < g:
                if key == 0.0:
                    shell += 1
                else:
                    tail += 1
    return shell, tail


@pytest.mark.parametrize("nd", [2, 3])
def test_cell_census_matches_brute_force(nd):
    rng = np.random.default_rng(5 + nd)
    shape = (9, 11) if nd == 2 else (5, 6, 7)
    spacing = (1.0, 1.5) if nd == 2 else (2.0, 1.5, 1.25)
    gamma = rng.uniform(0.0, 2.5, shape)
    gamma[rng.uniform(size=shape) < 0.3] = np.nan       # voxels below the cutoff
    gamma[(0,) * nd] = 0.0                               # gamma = 0 certifies nothing
    want = _brute_census(gamma, spacing, 2.0)
    got = bench.cell_census(torch.from_numpy(gamma), spacing, 2.0)
    assert tuple(int(x) for x in got) == want


def test_cell_census_empty_map():
    gamma = np.full((4, 5, 6), np.nan)
    assert tuple(bench.cell_census(torch.from_numpy(gamma), (1.0, 1.0, 1.0), 3.0)) == (0, 0)


def test_record_counters_reads_an_ncu_raw_csv(tmp_path, monkeypatch):
    # the layout of `ncu -i REPORT --page raw --csv`: a header row of metric
    # names, a row of units, then one row per captured launch
    csv_text = (
        '"ID","Kernel Name","gpu__time_duration.sum","dram__bytes_read.sum","dram__bytes_write.sum",'
        '"smsp__inst_executed.sum","smsp__thread_inst_executed_per_inst_executed.ratio",'
        '"sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active"\n'
        '"","","us","Mbyte","Kbyte","inst","","%"\n'
        '"0","void gk::k_shell<3, 4, false>(gk::Problem, CUtensorMap_st, int)","80","25.467904","0",'
        '"7,000,000","27.1","22.1"\n'
        '"1","void gk::k_walk<3, 2>(gk::Problem, CUtensorMap_st, int)","40","9","1",'
        '"3,000,000","20","30.5"\n')
    src = tmp_path / "raw.csv"
    src.write_text(csv_text)
    monkeypatch.setattr(bench, "COUNTERS_PATH", str(tmp_path / "counters.json"))
    out = bench.record_counters(str(src), "imrt_160", "test capture")
    assert set(out) == {"k_shell", "k_walk"}
    assert out["k_shell"]["dram_read_bytes"] == 25467904
    assert out["k_walk"]["warp_inst_per_launch"] == 3e6
    assert out["k_walk"]["fma_pipe_pct"] == 30.5
    assert out["k_walk"]["lane_efficiency"] == 20.0
    assert out["k_shell"]["ncu_duration_ns"] == 80000
    assert bench.recorded_traffic("k_walk", "imrt_160") == 9001000
    assert bench.recorded_traffic("k_walk", "plane_128") is None
