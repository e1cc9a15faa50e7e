"""Host logic of the periodic re-tuning (Sec. V-A3: the threshold is tuned
again every N iterations), with the GPU timing replaced by a stand-in."""
import types

import pytest

from paper_2401_05345_gb300 import autotune


def test_retunes_every_period_calls_per_key(monkeypatch):
    calls = []

    def fake_tune(vb, bg, dimg, candidates=None, reps=5, flush=None):
        calls.append(vb)
        return types.SimpleNamespace(best=f"best-{vb}-{len(calls)}")

    monkeypatch.setattr(autotune, "tune", fake_tune)
    at = autotune.Autotuner(period=3)
    got = [at.opts("a", "A", None, None) for _ in range(7)]
    # tuned at calls 0, 3 and 6 of key "a"; the choice is kept in between
    assert calls == ["A", "A", "A"]
    assert got == ["best-A-1"] * 3 + ["best-A-2"] * 3 + ["best-A-3"]
    # another key has its own count and choice
    assert at.opts("b", "B", None, None) == "best-B-4"
    assert at.opts("a", "A", None, None) == "best-A-3"
    assert calls == ["A", "A", "A", "B"]


def test_period_zero_tunes_once(monkeypatch):
    n = {"tunes": 0}

    def fake_tune(vb, bg, dimg, candidates=None, reps=5, flush=None):
        n["tunes"] += 1
        return types.SimpleNamespace(best="x")

    monkeypatch.setattr(autotune, "tune", fake_tune)
    at = autotune.Autotuner(period=0)
    for _ in range(10):
        assert at.opts("k", None, None, None) == "x"
    assert n["tunes"] == 1


def test_candidate_names_round_trip():
    for o in autotune.default_candidates():
        p = autotune.parse_opts_name(autotune.opts_name(o))
        assert autotune.opts_key(p) == autotune.opts_key(o)
