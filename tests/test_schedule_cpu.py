"""Host logic of the symmetric pair pass (csrc/sym_schedule.h), compiled on its own with g++ and
checked on the CPU: every unordered unit (target tile b, source tile t >= b) of the upper triangle is
covered exactly once, the source-partial slots of the units t > b are distinct and dense, row
segments are contiguous and in order, and (single suspension) the CTA runs have equal length up to
the last; (shares of the triangle among processes) the shares cover it once and read back exactly
the partials they wrote; (batched) no unit crosses a suspension and a suspension's lists do not depend on its
companions."""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1612_00474_gb300", "csrc")
TILE = 128


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("sched") / "schedule_dump")
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, os.path.join(HERE, "schedule_dump.cpp"), "-o", exe],
                   check=True)

    def run(*args):
        out = subprocess.run([exe, *map(str, args)], check=True, capture_output=True, text=True).stdout
        return json.loads(out)

    return run


def _segments(d):
    s = d["seg4"]
    return [tuple(s[4 * q:4 * q + 4]) for q in range(len(s) // 4)]


@pytest.mark.parametrize("N,sms", [(1, 152), (128, 152), (129, 152), (1000, 4), (65536, 152), (70000, 152)])
def test_single_schedule(dump, N, sms):
    d = dump("single", N, sms)
    nb = -(-N // TILE)
    segs = _segments(d)
    units = {}
    for q, (b, t0, t1, _) in enumerate(segs):
        assert 0 <= b <= t0 < t1 <= nb
        assert d["row_seg"][b] <= q < d["row_seg"][b + 1]
        for t in range(t0, t1):
            assert (b, t) not in units
            units[(b, t)] = q
    assert set(units) == {(b, t) for b in range(nb) for t in range(b, nb)}
    # row b's segments cover [b, nb) in order
    for b in range(nb):
        row = segs[d["row_seg"][b]:d["row_seg"][b + 1]]
        assert [s[1] for s in row] == [b] + [s[2] for s in row[:-1]] and row[-1][2] == nb
    # source-partial slots of the units t > b: distinct and 0 .. nb(nb-1)/2 - 1
    slots = sorted(d["col_start"][t] + b for (b, t) in units if t > b)
    assert slots == list(range(nb * (nb - 1) // 2))
    # CTAs: consecutive segment ranges covering all segments, equal unit counts except the last
    cta = [tuple(d["cta4"][4 * c:4 * c + 2]) for c in range(len(d["cta4"]) // 4)]
    assert cta[0][0] == 0 and cta[-1][1] == len(segs)
    assert all(a[1] == b[0] for a, b in zip(cta, cta[1:]))
    work = [sum(segs[q][2] - segs[q][1] for q in range(s0, s1)) for s0, s1 in cta]
    units_n = nb * (nb + 1) // 2
    L = -(-units_n // min(units_n, 60 * sms))  # run length; at most 60 x SMs runs
    assert len(cta) == -(-units_n // L) and work[0] == L
    assert len(set(work[:-1])) <= 1 and work[-1] <= work[0]


@pytest.mark.parametrize("N,sms,nparts", [(1000, 4, 2), (1000, 4, 3), (300, 152, 7), (65536, 152, 8),
                                          (70000, 152, 3), (129, 152, 5)])
def test_part_schedules_share_the_triangle(dump, N, sms, nparts):
    """The shares of rpb_mobility_apply_part: nparts contiguous unit ranges of (nearly) equal size that
    together cover every unit of the triangle exactly once; each share's CTA runs have equal length up
    to the last; row_seg indexes its own segments; col_rows[t] = [r0, r1) is exactly the set of rows
    r < t whose unit (r, t) the share holds (the reduce kernel reads those source partials and no
    other), so that the shares' partial products add up to the whole product."""
    nb = -(-N // TILE)
    units_n = nb * (nb + 1) // 2
    seen = {}
    sizes = []
    for p in range(nparts):
        d = dump("part", N, sms, p, nparts)
        sizes.append(d["u1"] - d["u0"])
        segs = _segments(d)
        mine = set()
        for q, (b, t0, t1, _) in enumerate(segs):
            assert 0 <= b <= t0 < t1 <= nb
            assert d["row_seg"][b] <= q < d["row_seg"][b + 1]
            for t in range(t0, t1):
                assert (b, t) not in seen
                seen[(b, t)] = p
                mine.add((b, t))
        # unit indices of the share: exactly [u0, u1) in row-major order
        idx = sorted(b * nb - b * (b - 1) // 2 + (t - b) for b, t in mine)
        assert idx == list(range(d["u0"], d["u1"]))
        cr = d["col_rows"]
        for t in range(nb):
            rows = sorted(b for (b, tt) in mine if tt == t and b < t)
            r0, r1 = cr[2 * t], cr[2 * t + 1]
            assert rows == list(range(r0, r1)), (p, t, rows, r0, r1)
        cta = [tuple(d["cta4"][4 * c:4 * c + 2]) for c in range(len(d["cta4"]) // 4)]
        if segs:
            assert cta[0][0] == 0 and cta[-1][1] == len(segs)
            work = [sum(segs[q][2] - segs[q][1] for q in range(s0, s1)) for s0, s1 in cta]
            assert len(set(work[:-1])) <= 1 and work[-1] <= work[0] and len(cta) <= 60 * sms
        else:
            assert cta == []
    assert set(seen) == {(b, t) for b in range(nb) for t in range(b, nb)}
    assert sum(sizes) == units_n and max(sizes) - min(sizes) <= 1


def test_whole_triangle_is_share_zero_of_one(dump):
    """The single-process schedule is share 0 of 1, and its col_rows read every row above the diagonal."""
    for N in (256, 1000, 65536):
        a, b = dump("single", N, 152), dump("part", N, 152, 0, 1)
        for k in ("cta4", "seg4", "row_seg", "col_start"):
            assert a[k] == b[k]
        nb = -(-N // TILE)
        assert b["col_rows"] == [x for t in range(nb) for x in ((0, t) if t > 0 else (0, 0))]


SIZES = [300, 64, 2100, 1, 1025, 129, 128]


def test_batch_schedule(dump):
    d = dump("batch", *SIZES)
    segs = _segments(d)
    nbs = [-(-n // TILE) for n in SIZES]
    assert d["ntiles"] == sum(nbs)
    units = set()
    for q, (b, t0, t1, k) in enumerate(segs):
        g, nb = d["tile0"][k], nbs[k]
        assert g <= b <= t0 < t1 <= g + nb and t1 - t0 <= 8
        assert d["tile_inst"][b] == k
        assert d["row_seg"][b] <= q < d["row_seg"][b + 1]
        for t in range(t0, t1):
            assert (b, t) not in units
            units.add((b, t))
    want = {(b, t) for k, nb in enumerate(nbs) for b in range(d["tile0"][k], d["tile0"][k] + nb)
            for t in range(b, d["tile0"][k] + nb)}
    assert units == want
    slots = sorted(d["col_start"][t] + b for (b, t) in units if t > b)
    assert slots == list(range(d["n_src_slots"]))
    # one CTA per segment, longest first
    order = d["cta_order"]
    assert sorted(order) == list(range(len(segs)))
    lens = [segs[q][2] - segs[q][1] for q in order]
    assert lens == sorted(lens, reverse=True)


def test_batch_schedule_independent_of_companions(dump):
    """The 1025-sphere suspension's segments, relative to its first tile, are the same alone and in
    a mix; so are its column slots relative to its first slot."""
    alone = dump("batch", 1025)
    mixed = dump("batch", 300, 2100, 1025, 64)
    k = 2
    g = mixed["tile0"][k]
    rel = [(b - g, t0 - g, t1 - g) for (b, t0, t1, kk) in _segments(mixed) if kk == k]
    assert rel == [(b, t0, t1) for (b, t0, t1, _) in _segments(alone)]
    nb = 9
    base = mixed["col_start"][g + 1] + g  # slot of unit (g, g + 1)
    for t in range(1, nb):
        for b in range(t):
            assert mixed["col_start"][g + t] + (g + b) - base == alone["col_start"][t] + b


@pytest.mark.parametrize("fp64", [0, 1])
def test_noalloc_partials_fit(fp64, tmp_path):
    """The allocation-free product's chunk plan keeps its partial sums (splits x 3N doubles) inside its
    fixed array for every N up to its limit and any SM count up to 1024, in chunks that cover the N
    sources exactly once (whole tiles in float32, multiples of 4 sources in float64)."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "schedule_dump")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "schedule_dump.cpp"), "-o", exe],
                   check=True)
    max_n = 16384                 # RPB_NOALLOC_MAX_N
    cap = 16 * 3 * max_n          # kNoAllocPartialElems
    out = subprocess.run([exe, "noalloc", str(max_n), "1024", str(cap), str(fp64)], check=True, capture_output=True,
                         text=True).stdout.split()
    assert out[-1] == "ok", out[:40]
