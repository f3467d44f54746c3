"""The oracle against its committed fixtures (tests/golden/oracle_fixtures.json,
written by tests/golden/make_golden.py from the oracle alone): a change to
the oracle's arithmetic must come with regenerated fixtures and a reason."""

import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def stored():
    with open(os.path.join(HERE, "golden", "oracle_fixtures.json")) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def fresh():
    import importlib.util

    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.fixtures()


def _close(a, b, rtol=1e-10):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return np.abs(a - b).max() <= rtol * max(1.0, np.abs(b).max())


def test_fixture_set_is_complete(stored, fresh):
    assert sorted(stored) == sorted(fresh)
    for k in stored:
        assert sorted(stored[k]) == sorted(fresh[k]), k


def test_oracle_reproduces_its_fixtures(stored, fresh):
    for name, entry in stored.items():
        for key, want in entry.items():
            got = fresh[name][key]
            if key == "inputs":
                assert got == want
            elif key == "iters":
                assert abs(got - want) <= 1, (name, got, want)  # rounding order may move the stop by one
            else:
                assert _close(got, want), (name, key)
