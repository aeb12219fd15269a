"""The autotuner's table on the host (no GPU): forms recorded by hand are
read back, written to the NTT_TUNE_DB file as one JSON object per line, and
read again by a fresh process."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nt():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2405_11353_gb300 as nt
    return nt


def _run(code, db):
    env = dict(os.environ, NTT_TUNE_DB=db, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    return r.stdout.strip()


def test_tune_table_set_get_persist(nt, tmp_path):
    db = str(tmp_path / "tune.jsonl")
    out = _run("import paper_2405_11353_gb300 as nt\n"
               "f = nt.NTT_ORDER_BITREV\n"
               "nt.ntt_tune_set(1 << 16, 32, f, 16, nt.NTT_FORM_WIDE, nt.NTT_FORM_SMALL)\n"
               "nt.ntt_tune_set(1 << 15, 4, f | nt.NTT_WORD64, 3, nt.NTT_FORM_STREAMED, nt.NTT_FORM_STREAMED)\n"
               "print(nt.ntt_tune_get(1 << 16, 32, f, 16), nt.ntt_tune_get(1 << 16, 32, f, 31, True),\n"
               "      nt.ntt_tune_get(1 << 16, 32, f, 32), nt.ntt_tune_get(1 << 16, 32, 0, 16))\n", db)
    # batches 16..31 share a bucket; batch 32 and natural order are other keys
    assert out == "1 0 -1 -1"
    lines = [json.loads(x) for x in open(db)]
    assert len(lines) == 2
    row = [x for x in lines if x["N"] == 1 << 16][0]
    assert (row["word_bytes"], row["L"], row["bitrev"], row["batch_log2"]) == (4, 32, 1, 4)
    assert (row["forward_form"], row["inverse_form"]) == (1, 0)
    out = _run("import paper_2405_11353_gb300 as nt\n"
               "print(nt.ntt_tune_get(1 << 15, 4, nt.NTT_ORDER_BITREV | nt.NTT_WORD64, 2, True),\n"
               "      nt.ntt_tune_get(1 << 16, 32, nt.NTT_ORDER_BITREV, 20))\n"
               "nt.ntt_tune_clear()\n"
               "print(nt.ntt_tune_get(1 << 16, 32, nt.NTT_ORDER_BITREV, 20))\n", db)
    assert out.split() == ["2", "1", "-1"]


def test_tune_set_rejects_bad_forms(nt):
    for fwd, inv, batch in [(5, 0, 4), (0, -1, 4), (0, 0, 0), (1, 5, 4)]:
        with pytest.raises(nt.NttError):
            nt.ntt_tune_set(1 << 16, 2, 0, batch, fwd, inv)


def test_tune_table_keys_twiddle_mode_and_reads_older_lines(nt, tmp_path):
    """NTT_TW_OTF plans have their own entries, written with a tw_otf field;
    lines without it (an older table) load as table-twiddle entries."""
    db = str(tmp_path / "tune.jsonl")
    with open(db, "w") as f:
        f.write('{"N": 32768, "word_bytes": 4, "L": 8, "reduction": 0, "bitrev": 1, "batch_log2": 2, '
                '"forward_form": 1, "inverse_form": 2, "forward_ms": [-1.0, -1.0, -1.0], '
                '"inverse_ms": [-1.0, -1.0, -1.0]}\n')
    out = _run("import paper_2405_11353_gb300 as nt\n"
               "f = nt.NTT_ORDER_BITREV\n"
               "print(nt.ntt_tune_get(1 << 15, 8, f, 4), nt.ntt_tune_get(1 << 15, 8, f, 4, True),\n"
               "      nt.ntt_tune_get(1 << 15, 8, f | nt.NTT_TW_OTF, 4))\n"
               "nt.ntt_tune_set(1 << 15, 8, f | nt.NTT_TW_OTF, 4, nt.NTT_FORM_SMALL, nt.NTT_FORM_WIDE)\n"
               "print(nt.ntt_tune_get(1 << 15, 8, f | nt.NTT_TW_OTF, 4, True), nt.ntt_tune_get(1 << 15, 8, f, 4))\n",
               db)
    assert out.split() == ["1", "2", "-1", "1", "1"]
    rows = [json.loads(x) for x in open(db)]
    assert sorted(r["tw_otf"] for r in rows) == [0, 1]


def test_split_table_set_get_persist(nt, tmp_path):
    """A shape's split (chunks of 2^s2 words) and radix are recorded by hand,
    refused where the size cannot take them, written as their own line, key
    the form entries, and are read by a fresh process; older lines without a
    split or radix field are forms of the default 256-word split, radix 16."""
    db = str(tmp_path / "tune.jsonl")
    with open(db, "w") as f:
        f.write('{"N": 65536, "word_bytes": 4, "L": 3, "reduction": 0, "bitrev": 1, "tw_otf": 0, '
                '"batch_log2": 2, "forward_form": 1, "inverse_form": 0, "forward_ms": [-1.0, -1.0, -1.0], '
                '"inverse_ms": [-1.0, -1.0, -1.0]}\n')
        f.write('{"N": 65536, "word_bytes": 4, "L": 5, "reduction": 0, "bitrev": 1, "tw_otf": 0, '
                '"chunk_log2": 7, "batch_log2": 2, "forward_form": 2, "inverse_form": 2, '
                '"forward_ms": [-1.0, -1.0, -1.0], "inverse_ms": [-1.0, -1.0, -1.0]}\n')
    out = _run("import paper_2405_11353_gb300 as nt\n"
               "f = nt.NTT_ORDER_BITREV\n"
               "print(*nt.ntt_tune_get_split(1 << 16, 3, f), nt.ntt_tune_get(1 << 16, 3, f, 4))\n"
               "nt.ntt_tune_set_split(1 << 16, 3, f, 9, 3)\n"
               "print(*nt.ntt_tune_get_split(1 << 16, 3, f), nt.ntt_tune_get(1 << 16, 3, f, 4))\n"
               "nt.ntt_tune_set(1 << 16, 3, f, 4, nt.NTT_FORM_SMALL, nt.NTT_FORM_SMALL)\n"
               "print(nt.ntt_tune_get(1 << 16, 3, f, 4, True))\n"
               "nt.ntt_tune_set_split(1 << 16, 5, f, 7, 4)\n"
               "print(nt.ntt_tune_get(1 << 16, 5, f, 4))\n"
               "bad = 0\n"
               "for args in ((1 << 17, 3, f, 7, 4), (1 << 15, 3, f, 10, 4), (1 << 16, 3, f | nt.NTT_TW_OTF, 7, 4),\n"
               "             (1 << 16, 3, f | nt.NTT_TW_OTF, 8, 3), (1 << 16, 3, f, 8, 5), (1000, 3, f, 8, 4),\n"
               "             (1 << 16, 0, f, 8, 4)):\n"
               "    try:\n"
               "        nt.ntt_tune_set_split(*args)\n"
               "    except nt.NttError:\n"
               "        bad += 1\n"
               "print(bad)\n", db)
    assert out.split() == ["-1", "-1", "1", "9", "3", "-1", "0", "2", "7"]
    rows = [json.loads(x) for x in open(db)]
    assert sorted((r["L"], r["split_log2"], r["radix_log2"]) for r in rows if "split_log2" in r) == [
        (3, 9, 3), (5, 7, 4)]
    forms = sorted((r["L"], r["chunk_log2"], r["radix_log2"], r["forward_form"]) for r in rows
                   if "chunk_log2" in r)
    assert forms == [(3, 8, 4, 1), (3, 9, 3, 0), (5, 7, 4, 2)]
    out = _run("import paper_2405_11353_gb300 as nt\n"
               "f = nt.NTT_ORDER_BITREV\n"
               "print(*nt.ntt_tune_get_split(1 << 16, 3, f), nt.ntt_tune_get(1 << 16, 3, f, 4))\n"
               "nt.ntt_tune_clear()\n"
               "print(*nt.ntt_tune_get_split(1 << 16, 3, f))\n", db)
    assert out.split() == ["9", "3", "0", "-1", "-1"]


def test_shuffle_forms_set_get_persist(nt, tmp_path):
    """The shuffle forms (3, 4) are recorded, written with five per-form
    times, and read back by a fresh process beside a three-time line."""
    db = str(tmp_path / "tune.jsonl")
    with open(db, "w") as f:
        f.write('{"N": 65536, "word_bytes": 4, "L": 7, "reduction": 0, "bitrev": 1, "tw_otf": 0, '
                '"chunk_log2": 8, "radix_log2": 4, "batch_log2": 3, "forward_form": 2, "inverse_form": 1, '
                '"forward_ms": [-1.0, -1.0, -1.0], "inverse_ms": [-1.0, -1.0, -1.0]}\n')
    out = _run("import paper_2405_11353_gb300 as nt\n"
               "f = nt.NTT_ORDER_BITREV\n"
               "nt.ntt_tune_set(1 << 16, 6, f, 4, nt.NTT_FORM_SMALL_SHFL, nt.NTT_FORM_WIDE_SHFL)\n"
               "print(nt.ntt_tune_get(1 << 16, 6, f, 4), nt.ntt_tune_get(1 << 16, 6, f, 4, True),\n"
               "      nt.ntt_tune_get(1 << 16, 7, f, 8))\n", db)
    assert out.split() == ["3", "4", "2"]
    rows = [json.loads(x) for x in open(db)]
    row = [r for r in rows if r["L"] == 6][0]
    assert (row["forward_form"], row["inverse_form"]) == (3, 4)
    assert len(row["forward_ms"]) == 5 and len(row["inverse_ms"]) == 5
    out = _run("import paper_2405_11353_gb300 as nt\n"
               "f = nt.NTT_ORDER_BITREV\n"
               "print(nt.ntt_tune_get(1 << 16, 6, f, 4), nt.ntt_tune_get(1 << 16, 6, f, 4, True),\n"
               "      nt.ntt_tune_get(1 << 16, 7, f, 8, True))\n", db)
    assert out.split() == ["3", "4", "1"]
