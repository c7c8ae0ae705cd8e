"""The autotuner's host table (no GPU work): classes by log2 of n and of the mean row
length, record/lookup, save/load round trip, merge, and rejection of malformed files."""
import pytest


@pytest.fixture()
def S():
    from paper_2102_08505_gb300 import sp2ell
    sp2ell.sp2_tune_clear()
    yield sp2ell
    sp2ell.sp2_tune_clear()


def test_classes_and_lookup(S):
    assert S.sp2_tune_lookup(152, S.SP2_F64, 262144, 138.6) == -1
    S.sp2_tune_record(152, S.SP2_F64, 262144, 138.6, 4, 34.3)
    # same class: n in [2^18, 2^19), mean row length in [128, 256)
    assert S.sp2_tune_lookup(152, S.SP2_F64, 300000, 200.0) == 4
    assert S.sp2_tune_lookup(152, S.SP2_F64, 262143, 138.6) == -1   # other n class
    assert S.sp2_tune_lookup(152, S.SP2_F64, 262144, 127.9) == -1   # other width class
    assert S.sp2_tune_lookup(152, S.SP2_F32, 262144, 138.6) == -1   # other dtype
    assert S.sp2_tune_lookup(148, S.SP2_F64, 262144, 138.6) == -1   # other device class
    S.sp2_tune_record(152, S.SP2_F64, 262144, 150.0, 2, 30.0)       # replaces the entry
    assert S.sp2_tune_lookup(152, S.SP2_F64, 262144, 138.6) == 2 and S.sp2_tune_size() == 1
    with pytest.raises(S.Sp2Error):
        S.sp2_tune_record(152, S.SP2_F64, 1000, 10.0, 0, 1.0)  # 0 (automatic) is not a variant
    with pytest.raises(S.Sp2Error):
        S.sp2_tune_record(0, S.SP2_F64, 1000, 10.0, 4, 1.0)


def test_save_load_round_trip(S, tmp_path):
    S.sp2_tune_record(152, S.SP2_F64, 262144, 138.6, 4, 34.3)
    S.sp2_tune_record(152, S.SP2_F32, 131072, 190.0, 3, 12.5)
    S.sp2_tune_record(152, S.SP2_F32, 1 << 20, 300.0, 11, 80.0)
    f = tmp_path / "tune.txt"
    S.sp2_tune_save(f)
    lines = f.read_text().splitlines()
    assert lines[0].startswith("# sp2ell spgemm tuning v1")
    assert lines[1:] == ["152 0 18 7 4 34.3", "152 1 17 7 3 12.5", "152 1 20 8 11 80"]
    S.sp2_tune_clear()
    assert S.sp2_tune_size() == 0
    S.sp2_tune_load(f)
    assert S.sp2_tune_size() == 3
    assert S.sp2_tune_lookup(152, S.SP2_F32, 131072, 190.0) == 3
    # load merges: an entry replaces its class, others stay
    S.sp2_tune_record(152, S.SP2_F64, 262144, 138.6, 1, 50.0)
    S.sp2_tune_record(152, S.SP2_F64, 1024, 20.0, 10, 0.1)
    S.sp2_tune_load(f)
    assert S.sp2_tune_lookup(152, S.SP2_F64, 262144, 138.6) == 4 and S.sp2_tune_size() == 4


def test_malformed_files_are_rejected(S, tmp_path):
    bad = [
        "152 0 18 7 4 34.3\n",                                          # no header
        "# sp2ell spgemm tuning v1\n152 0 18 7 13 1.0\n",               # 13 is not a variant
        "# sp2ell spgemm tuning v1\n152 2 18 7 4 1.0\n",                # unknown dtype
        "# sp2ell spgemm tuning v1\n152 0 18\n",                        # short line
    ]
    for k, text in enumerate(bad):
        f = tmp_path / ("bad%d.txt" % k)
        f.write_text(text)
        with pytest.raises(S.Sp2Error) as e:
            S.sp2_tune_load(f)
        assert e.value.code == S.SP2E_ARG
        assert S.sp2_tune_size() == 0
    with pytest.raises(S.Sp2Error):
        S.sp2_tune_load(tmp_path / "missing.txt")
