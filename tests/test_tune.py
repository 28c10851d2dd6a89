"""Host logic of the tuning table (gw_tune_*): entries, precedence, checks,
candidates and the table file.  No GPU: these entry points make no CUDA call."""
import pytest

from paper_2404_08970_gb300 import _lib as L

SK = L.GW_TUNE_SINKHORN
F32, F64 = L.GW_F32, L.GW_F64
ROW_LENGTHS = [1, 7, 255, 256, 257, 512, 513, 900, 1024, 1025, 2048, 2049, 4096, 4097, 5000, 8192, 8193,
               9216, 9217, 12000, 16384]


@pytest.fixture(autouse=True)
def clean_table():
    L.gw_tune_clear()
    yield
    L.gw_tune_clear()


def cover(config):
    nw, vpt, _ = L.gw_tune_shape(SK, config)
    return 32 * nw * vpt


@pytest.mark.parametrize("dtype", [F32, F64])
def test_builtin_choice_covers_the_row(dtype):
    for m in ROW_LENGTHS:
        c = L.gw_tune_config(SK, dtype, m)
        assert c >= 0 and cover(c) >= m, (m, c)


@pytest.mark.parametrize("dtype", [F32, F64])
def test_candidates(dtype):
    esz = 4 if dtype == F32 else 8
    for m in ROW_LENGTHS:
        cands = L.gw_tune_candidates(SK, dtype, m)
        assert cands[0] == L.gw_tune_config(SK, dtype, m)
        assert len(set(cands)) == len(cands)
        base = cover(cands[0])
        for c in cands:
            nw, vpt, ng = L.gw_tune_shape(SK, c)
            assert m <= 32 * nw * vpt <= 4 * base, (m, c)
            assert 32 * nw * ng <= 1024 and (vpt * esz) % 16 == 0, (m, c)
            # A candidate is accepted as an entry for exactly this row length.
            L.gw_tune_set(SK, dtype, m, m, c)
            assert L.gw_tune_config(SK, dtype, m) == c


def test_entries_and_precedence():
    default_800 = L.gw_tune_config(SK, F32, 800)
    L.gw_tune_set(SK, F32, 700, 900, 21)
    assert L.gw_tune_config(SK, F32, 800) == 21
    assert L.gw_tune_config(SK, F32, 699) == L.gw_tune_config(SK, F32, 600)
    assert L.gw_tune_config(SK, F32, 901) == default_800   # same built-in range (513..1024)
    assert L.gw_tune_config(SK, F64, 800) != 21            # per dtype
    L.gw_tune_set(SK, F32, 800, 800, 2)                    # a later entry wins
    assert L.gw_tune_config(SK, F32, 800) == 2
    assert L.gw_tune_config(SK, F32, 799) == 21
    L.gw_tune_clear()
    assert L.gw_tune_config(SK, F32, 800) == default_800


@pytest.mark.parametrize("args", [
    (1, F32, 1, 512, 0),        # unknown kernel
    (SK, 7, 1, 512, 0),         # unknown dtype
    (SK, F32, 0, 512, 0),       # empty / non-positive range
    (SK, F32, 600, 500, 1),
    (SK, F32, 1, 20000, 6),     # beyond the solver's 16384 columns
    (SK, F32, 1, 2000, 21),     # 4 x 8 x 32 = 1024 columns do not cover 2000
    (SK, F64, 1, 256, 20),      # a float configuration for double rows
    (SK, F32, 1, 256, 99),      # no such configuration
])
def test_invalid_entries_rejected(args):
    with pytest.raises(L.GWError) as e:
        L.gw_tune_set(*args)
    assert e.value.status == L.GW_ERR_INVALID
    assert L.gw_tune_config(SK, F32, 300) == L.gw_tune_candidates(SK, F32, 300)[0]


def test_queries_reject_bad_arguments():
    assert L.gw_tune_config(SK, F32, 0) == -1
    assert L.gw_tune_config(SK, F32, 16385) == -1
    assert L.gw_tune_config(3, F32, 100) == -1
    with pytest.raises(L.GWError):
        L.gw_tune_candidates(SK, 5, 100)
    with pytest.raises(L.GWError):
        L.gw_tune_shape(SK, 99)


def test_table_file(tmp_path):
    good = tmp_path / "tune_table.txt"
    good.write_text("# kernel dtype m_lo m_hi config\n"
                    "\n"
                    f"{SK} {F32} 513 1024 21   # 4 x 8 x 4\n"
                    f"   {SK} {F64} 1 256 30\n")
    L.gw_tune_load(str(good))
    assert L.gw_tune_config(SK, F32, 600) == 21
    assert L.gw_tune_config(SK, F64, 100) == 30

    L.gw_tune_clear()
    bad = tmp_path / "bad.txt"
    bad.write_text(f"{SK} {F32} 513 1024 21\n"
                   f"{SK} {F32} 1 2000 21\n"       # does not cover 2000 columns
                   f"{SK} {F64} 1 256 30\n")
    with pytest.raises(L.GWError):
        L.gw_tune_load(str(bad))
    assert L.gw_tune_config(SK, F32, 600) == 21      # the line before the bad one stays
    assert L.gw_tune_config(SK, F64, 100) != 30      # the lines after it are not read

    L.gw_tune_clear()
    junk = tmp_path / "junk.txt"
    junk.write_text(f"{SK} {F32} 513 1024\n")
    with pytest.raises(L.GWError):
        L.gw_tune_load(str(junk))
    with pytest.raises(L.GWError):
        L.gw_tune_load(str(tmp_path / "missing.txt"))


def test_sweep_ranges_and_table_round_trip(tmp_path):
    """The sweep's half ranges tile each built-in range, and the table it
    writes is read back by gw_tune_load with the same entries."""
    from paper_2404_08970_gb300 import tune
    for dtype, ranges in tune.RANGES.items():
        prev_hi = 0
        for lo, hi in ranges:
            assert lo == prev_hi + 1
            assert L.gw_tune_config(SK, dtype, lo) == L.gw_tune_config(SK, dtype, hi)   # one built-in choice
            parts = tune.halves(lo, hi)
            assert parts[0][0] == lo and parts[-1][1] == hi
            assert all(b + 1 == c for (_, b), (c, _) in zip(parts, parts[1:]))
            prev_hi = hi
        # The longest row the solver takes in this dtype.
        assert prev_hi == (16384 if dtype == F32 else 10240)
    entries = [(F32, 513, 768, 21, {1: 0.5, 21: 0.4}), (F32, 769, 1024, 1, {1: 0.5, 21: 0.6}),
               (F64, 1, 128, 30, {10: 1.0, 30: 0.9})]
    path = tmp_path / "tune_table.txt"
    tune.write_table(str(path), entries, ["dtype 0 m 1024 config 2: plan differs by 1.00e-02; dropped"], 2048, 3,
                     "test device")
    L.gw_tune_load(str(path))
    assert L.gw_tune_config(SK, F32, 600) == 21
    assert L.gw_tune_config(SK, F32, 900) == 1
    assert L.gw_tune_config(SK, F64, 100) == 30


def test_committed_table_loads_and_is_consistent():
    """The committed table (read at context creation) loads, has one entry per
    half range of the sweep, and each entry names a candidate of its longest
    row (so it covers every row of its range)."""
    import os
    from paper_2404_08970_gb300 import tune
    path = os.path.join(os.path.dirname(os.path.abspath(L.__file__)), "tune_table.txt")
    rows = []
    for line in open(path):
        body = line.split("#")[0].split()
        if body:
            rows.append(tuple(int(x) for x in body))
    want = [(SK, dt, a, b) for dt, ranges in tune.RANGES.items() for lo, hi in ranges for a, b in tune.halves(lo, hi)]
    assert sorted(r[:4] for r in rows) == sorted(want)
    L.gw_tune_load(path)
    for kernel, dt, lo, hi, cfg in rows:
        assert L.gw_tune_config(kernel, dt, lo) == cfg and L.gw_tune_config(kernel, dt, hi) == cfg
        assert cfg in L.gw_tune_candidates(kernel, dt, hi), (lo, hi, cfg)
        assert cover(cfg) >= hi
