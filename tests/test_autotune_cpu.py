"""The autotuned launch table's lookup (no GPU): a (d, density, states)
shape finds its bucket's tile rows and grid cap; a table of the older form
(no state buckets, no grid cap) still gives its rows; shapes outside every
bucket, and rows a width cannot stage, fall back to the library default."""
import json

from paper_2407_11388_b300 import autotune


def _write(tmp_path, entries):
    p = tmp_path / "table.json"
    p.write_text(json.dumps({"version": 2, "entries": entries}))
    return str(p)


def test_lookup_by_state_bucket(tmp_path):
    path = _write(tmp_path, [
        {"d_lo": 17, "d_hi": 24, "dens_lo": 0.6, "dens_hi": 1.0, "st_lo": 1, "st_hi": 1,
         "rows": 4, "max_ctas": 74},
        {"d_lo": 17, "d_hi": 24, "dens_lo": 0.6, "dens_hi": 1.0, "st_lo": 2, "st_hi": 1 << 30,
         "rows": 8, "max_ctas": None},
    ])
    assert autotune.table_choice(20, 1.0, 1, path) == (4, 74)
    assert autotune.table_choice(24, 0.8, 32, path) == (8, None)
    assert autotune.table_choice(24, 0.3, 32, path) == (None, None)   # no density bucket
    assert autotune.table_choice(30, 0.8, 1, path) == (None, None)    # no d bucket


def test_older_table_and_rows_that_do_not_fit(tmp_path):
    path = _write(tmp_path, [
        {"d_lo": 25, "d_hi": 32, "dens_lo": 0.0, "dens_hi": 1.0, "rows": 32},
        {"d_lo": 1, "d_hi": 8, "dens_lo": 0.0, "dens_hi": 1.0, "rows": 32},
    ])
    # 32 rows of width 32 take 128 KiB: more than a stage holds
    assert autotune.table_choice(32, 0.9, 1, path) == (None, None)
    assert autotune.table_choice(8, 0.5, 64, path) == (32, None)
    assert autotune.admissible_rows(32) == [2, 4, 8]
    assert autotune.admissible_rows(8) == [2, 4, 8, 16, 32]


def test_plan_entries_are_looked_up_apart(tmp_path):
    path = _write(tmp_path, [
        {"kind": "plan", "d_lo": 1, "d_hi": 8, "dens_lo": 0.0, "dens_hi": 1.0, "rows": 32},
        {"d_lo": 1, "d_hi": 8, "dens_lo": 0.0, "dens_hi": 1.0, "st_lo": 2, "st_hi": 1 << 30,
         "rows": 8, "max_ctas": None},
    ])
    assert autotune.table_choice(6, 0.5, 64, path, kind="plan") == (32, None)
    assert autotune.table_choice(6, 0.5, 64, path) == (8, None)
    assert autotune.table_choice(6, 0.5, 1, path) == (None, None)


def test_relation_layout_entries(tmp_path):
    """An entry's packed flag is looked up with its rows; the rows of a packed
    entry are checked against the packed tile size (16 rows of d = 20 fit a
    stage only packed)."""
    path = _write(tmp_path, [
        {"d_lo": 17, "d_hi": 24, "dens_lo": 0.6, "dens_hi": 1.0, "st_lo": 1, "st_hi": 1,
         "rows": 16, "max_ctas": None, "packed": True},
        {"d_lo": 17, "d_hi": 24, "dens_lo": 0.6, "dens_hi": 1.0, "st_lo": 2, "st_hi": 1 << 30,
         "rows": 8, "max_ctas": None, "packed": False},
    ])
    assert autotune.table_packed(20, 0.9, 1, path) is True
    assert autotune.table_packed(20, 0.9, 32, path) is False
    assert autotune.table_packed(20, 0.3, 1, path) is False          # no density bucket
    assert autotune.table_choice(20, 0.9, 1, path, packed=True) == (16, None)
    assert autotune.table_choice(20, 0.9, 1, path, packed=False) == (None, None)
    assert autotune.admissible_rows(20) == [2, 4, 8]
    assert autotune.admissible_rows(20, packed=True) == [2, 4, 8, 16]
    assert autotune.admissible_rows(12, packed=True) == [2, 4, 8, 16, 32]
    assert autotune.words_per_relation(24, packed=True) == 18
    assert autotune.words_per_relation(30, packed=True) == 32


def test_one_state_entries_split_by_size(tmp_path):
    """One-state entries may carry a constraint-count range: the lookup takes
    the entry whose range holds the network's m (and, without m, the first
    entry of the bucket)."""
    path = _write(tmp_path, [
        {"d_lo": 17, "d_hi": 20, "dens_lo": 0.6, "dens_hi": 1.0, "st_lo": 1, "st_hi": 1,
         "m_lo": 0, "m_hi": 99999, "rows": 8, "max_ctas": None, "packed": False},
        {"d_lo": 17, "d_hi": 20, "dens_lo": 0.6, "dens_hi": 1.0, "st_lo": 1, "st_hi": 1,
         "m_lo": 100000, "m_hi": 1 << 62, "rows": 16, "max_ctas": None, "packed": True},
    ])
    assert autotune.table_choice(20, 1.0, 1, path, packed=False, m=5000) == (8, None)
    assert autotune.table_packed(20, 1.0, 1, path, m=5000) is False
    assert autotune.table_packed(20, 1.0, 1, path, m=124750) is True
    assert autotune.table_choice(20, 1.0, 1, path, packed=True, m=124750) == (16, None)
    assert autotune.table_choice(20, 1.0, 1, path, packed=False, m=124750) == (None, None)
    assert autotune.table_choice(20, 1.0, 1, path) == (8, None)
