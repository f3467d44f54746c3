"""CPU tests of the autotuner's cache (host code only, through the C ABI):
the key names (kernel, format, Naik storage, right-hand sides, extents);
put/get; a JSON round trip through a file; malformed or missing files leave
the cache unchanged; a fresh process picks the file named by STAG_TUNE_CACHE
up on first use and rewrites it on a new entry."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def stag():
    import paper_1712_00143_gb300 as s

    s.stag_tune_cache_clear()
    yield s
    s.stag_tune_cache_clear()


def test_keys_name_every_field(stag):
    k = stag.stag_tune_key("dslash_mrhs", "fp32", 6, 4, (32, 32, 32, 32))
    assert k == "dslash_mrhs/fp32/nl6/n4/32x32x32x32"
    others = {
        stag.stag_tune_key("dslash_mrhs", "fx16", 6, 4, (32, 32, 32, 32)),
        stag.stag_tune_key("dslash_mrhs", "fp32", 9, 4, (32, 32, 32, 32)),
        stag.stag_tune_key("dslash_mrhs", "fp32", 6, 8, (32, 32, 32, 32)),
        stag.stag_tune_key("dslash_mrhs", "fp32", 6, 4, (24, 24, 24, 48)),
        stag.stag_tune_key("dslash_mrhs", "fp32", 6, 4, (32, 32, 48, 32)),
        stag.stag_tune_key("dslash_df", "df64", 9, 4, (32, 32, 32, 32)),
    }
    assert k not in others and len(others) == 6


def test_put_get_and_file_round_trip(stag, tmp_path):
    k1 = stag.stag_tune_key("dslash_mrhs", "fp32", 6, 4, (32, 32, 32, 32))
    k2 = stag.stag_tune_key("dslash_mrhs", "fp32", 6, 8, (16, 16, 16, 16))
    assert stag.stag_tune_cache_size() == 0
    assert stag.stag_tune_cache_get(k1) == (-1, 0.0)
    stag.stag_tune_cache_put(k1, 3, 104.5)
    stag.stag_tune_cache_put(k2, 1, 55.25)
    stag.stag_tune_cache_put(k2, 4, 50.0)  # replaces
    assert stag.stag_tune_cache_get(k1) == (3, 104.5)
    assert stag.stag_tune_cache_get(k2) == (4, 50.0)
    path = tmp_path / "tune.json"
    stag.stag_tune_cache_save(str(path))
    d = json.loads(path.read_text())
    assert d["version"] == 1 and d["entries"][k1] == {"variant": 3, "us": 104.5}
    stag.stag_tune_cache_clear()
    assert stag.stag_tune_cache_size() == 0
    stag.stag_tune_cache_load(str(path))
    assert stag.stag_tune_cache_size() == 2
    assert stag.stag_tune_cache_get(k1) == (3, 104.5) and stag.stag_tune_cache_get(k2) == (4, 50.0)


@pytest.mark.parametrize(
    "text",
    [
        "",
        "{}",
        '{"version": 2, "entries": {}}',
        '{"version": 1, "entries": {"k": {"variant": 1}}}',
        '{"version": 1, "entries": {"k": {"variant": 1.5, "us": 3}}}',
        '{"version": 1, "entries": {"k": {"variant": 1, "us": 3}}',
        '{"version": 1, "entries": {"k": {"variant": 1, "us": 3}}} trailing',
    ],
)
def test_malformed_files_are_refused(stag, tmp_path, text):
    stag.stag_tune_cache_put("keep/me", 2, 1.0)
    path = tmp_path / "bad.json"
    path.write_text(text)
    with pytest.raises(stag.StagError):
        stag.stag_tune_cache_load(str(path))
    assert stag.stag_tune_cache_size() == 1 and stag.stag_tune_cache_get("keep/me") == (2, 1.0)
    with pytest.raises(stag.StagError):
        stag.stag_tune_cache_load(str(tmp_path / "missing.json"))
    with pytest.raises(stag.StagError):
        stag.stag_tune_cache_put("k", -1, 1.0)


def test_environment_file_is_read_and_rewritten(tmp_path):
    path = tmp_path / "env.json"
    path.write_text('{"version": 1, "entries": {"dslash_mrhs/fp32/nl6/n4/8x8x8x8": {"variant": 5, "us": 7.5}}}')
    code = (
        "import paper_1712_00143_gb300 as s\n"
        "print(s.stag_tune_cache_get('dslash_mrhs/fp32/nl6/n4/8x8x8x8'))\n"
        "s.stag_tune_cache_put('dslash_mrhs/fx16/nl6/n2/8x8x8x8', 2, 3.0)\n"
    )
    env = dict(os.environ, STAG_TUNE_CACHE=str(path))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "(5, 7.5)"
    d = json.loads(path.read_text())
    assert d["entries"]["dslash_mrhs/fx16/nl6/n2/8x8x8x8"] == {"variant": 2, "us": 3.0}
    assert d["entries"]["dslash_mrhs/fp32/nl6/n4/8x8x8x8"] == {"variant": 5, "us": 7.5}
