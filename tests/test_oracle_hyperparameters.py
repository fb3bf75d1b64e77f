"""The hyper-parameter table (Section V) against every place that turns q into a parameter:
the oracles (pruning, SH compaction, codec) and the package's host-side parameter functions.
The table is the fixture tests/golden/hyperparameters.txt, transcribed from the paper."""
import math
import os

import pytest

from oracle import codec as ocodec
from oracle import prune as oprune
from oracle import sh_compact as oshc

HERE = os.path.dirname(os.path.abspath(__file__))
QS = (0.0, 0.1, 0.3, 0.5, 0.77, 1.0)


def _table() -> dict:
    out = {}
    with open(os.path.join(HERE, "golden", "hyperparameters.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                name, expr = line.split(None, 1)
                out[name] = expr
    return out


def _value(expr: str, q: float) -> float:
    env = {"q": q, "sigmoid": lambda x: 1.0 / (1.0 + math.exp(-x)), "__builtins__": {}}
    return float(eval(expr, env))  # the fixture's own arithmetic expressions, nothing else


def test_fixture_lists_the_whole_table():
    assert set(_table()) == {"lambda", "alpha", "dmse_max", "beta", "gamma", "sf_sh", "sf_opacity", "sf_rotation",
                             "sf_scale", "iterations"}


@pytest.mark.parametrize("q", QS)
def test_oracles_follow_the_table(q):
    t = _table()
    want = {k: _value(e, q) for k, e in t.items()}
    sh = oshc.params(q)
    co = ocodec.params(q)
    got = {"lambda": sh["lam"], "alpha": sh["alpha"], "sf_sh": co["sf_sh"], "dmse_max": oprune.dmse_max(q),
           "beta": co["beta"], "gamma": co["gamma"], "sf_opacity": co["sf_opacity"],
           "sf_rotation": co["sf_rotation"], "sf_scale": co["sf_scale"],
           "iterations": float(oprune.ITERATIONS_DEFAULT)}
    assert sh["sf"] == pytest.approx(want["sf_sh"], rel=1e-15)  # the compaction's quantiser is the codec's
    for k in want:
        assert got[k] == pytest.approx(want[k], rel=1e-15), k


@pytest.mark.parametrize("q", QS)
def test_package_parameter_functions_follow_the_table(q):
    from paper_2601_14821_gb300 import codec, prune, sh_compact

    want = {k: _value(e, q) for k, e in _table().items()}
    sh = sh_compact.params(q)
    co = codec.params(q)
    assert sh["lam"] == pytest.approx(want["lambda"], rel=1e-15)
    assert sh["alpha"] == pytest.approx(want["alpha"], rel=1e-15)
    assert sh["sf"] == pytest.approx(want["sf_sh"], rel=1e-15)
    assert prune.dmse_max(q) == pytest.approx(want["dmse_max"], rel=1e-15)
    assert prune.ITERATIONS_DEFAULT == want["iterations"]
    for k in ("sf_sh", "sf_opacity", "sf_rotation", "sf_scale", "beta", "gamma"):
        assert co[k] == pytest.approx(want[k], rel=1e-15), k
