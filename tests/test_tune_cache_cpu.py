"""The tuners' cache on the host: entries keyed by device model and size class, saved as JSON
and loaded back (also from the POLYMUL_TUNE_CACHE environment variable in a fresh process).
No kernel runs here."""
import json
import os
import subprocess
import sys

import pytest

from paper_1402_0264_gb300 import build as pbuild
from paper_1402_0264_gb300 import polymul as pm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = pm.P_DEFAULT


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return pm.lib()


def _entries():
    return [
        {"device": "NVIDIA GB300", "sms": 152, "form": 1, "p_class": 0, "bucket1": 14, "bucket2": 14, "s": 8,
         "q": 0, "ms": 0.049},
        {"device": "NVIDIA GB300", "sms": 152, "form": 2, "p_class": 0, "bucket1": 11, "bucket2": 12, "s": 4,
         "q": 512, "ms": 0.18},
        {"device": "Other \"GPU\"", "sms": 80, "form": 1, "p_class": 1, "bucket1": 10, "bucket2": 3, "s": 2,
         "q": 0, "ms": 1.5},
    ]


def test_save_load_round_trip(lib, tmp_path):
    src = tmp_path / "in.json"
    src.write_text(json.dumps({"version": 1, "entries": _entries()}))
    pm.tune_clear()
    assert pm.tune_lookup("NVIDIA GB300", 152, pm.PM_TUNE_PLAIN, P, 16384, 16384) == (0, 0)
    pm.tune_load(str(src))
    # buckets: floor(log2) of the longer and shorter length (plain), of max_deg + 1 and batch (batched)
    assert pm.tune_lookup("NVIDIA GB300", 152, pm.PM_TUNE_PLAIN, P, 16384, 20000) == (8, 0)
    assert pm.tune_lookup("NVIDIA GB300", 152, pm.PM_TUNE_PLAIN, P, 30000, 16384) == (8, 0)   # operands in any order
    assert pm.tune_lookup("NVIDIA GB300", 152, pm.PM_TUNE_BATCHED, P, 2049, 4096) == (4, 512)
    assert pm.tune_lookup("NVIDIA GB300", 152, pm.PM_TUNE_BATCHED, P, 2049, 8192) == (0, 0)   # another batch bucket
    assert pm.tune_lookup("NVIDIA GB300", 148, pm.PM_TUNE_PLAIN, P, 16384, 16384) == (0, 0)   # another SM count
    assert pm.tune_lookup("NVIDIA GB300", 152, pm.PM_TUNE_PLAIN, 2**29 + 11, 16384, 16384) == (0, 0)  # p class
    assert pm.tune_lookup('Other "GPU"', 80, pm.PM_TUNE_PLAIN, 2**29 + 11, 1500, 9) == (2, 0)
    out = tmp_path / "out.json"
    pm.tune_save(str(out))
    saved = json.loads(out.read_text())
    assert saved["version"] == 1
    key = lambda e: (e["device"], e["sms"], e["form"], e["p_class"], e["bucket1"], e["bucket2"])
    assert sorted((key(e), e["s"], e["q"]) for e in saved["entries"]) == \
        sorted((key(e), e["s"], e["q"]) for e in _entries())
    pm.tune_clear()
    pm.tune_load(str(out))
    assert pm.tune_lookup("NVIDIA GB300", 152, pm.PM_TUNE_BATCHED, P, 2049, 4096) == (4, 512)
    pm.tune_clear()


def test_bad_files_are_refused(lib, tmp_path):
    pm.tune_clear()
    bad = tmp_path / "bad.json"
    for text in ("", "{", '{"version": 1}', '{"entries": [{"device": "x", "sms": 1}]}', "[1, 2]",
                 '{"entries": [{"device": "x", "sms": 1, "form": 7, "p_class": 0, "bucket1": 1, "bucket2": 1, "s": 2}]}'):
        bad.write_text(text)
        with pytest.raises(pm.PolymulError) as ei:
            pm.tune_load(str(bad))
        assert ei.value.code == 1, text
    with pytest.raises(pm.PolymulError):
        pm.tune_load(str(tmp_path / "missing.json"))
    with pytest.raises(pm.PolymulError):
        pm.tune_save(str(tmp_path / "no_such_dir" / "x.json"))
    assert lib.polymul_tune_lookup(b"x", 1, 9, P, 1, 1, None, None) == 1
    assert pm.tune_lookup("NVIDIA GB300", 152, pm.PM_TUNE_PLAIN, P, 16384, 16384) == (0, 0)


def test_environment_file_is_loaded_in_a_fresh_process(tmp_path):
    src = tmp_path / "env.json"
    src.write_text(json.dumps({"version": 1, "entries": _entries()}))
    code = ("from paper_1402_0264_gb300 import polymul as pm; "
            "print(pm.tune_lookup('NVIDIA GB300', 152, pm.PM_TUNE_BATCHED, pm.P_DEFAULT, 2049, 4096))")
    env = dict(os.environ, POLYMUL_TUNE_CACHE=str(src))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "(4, 512)"
