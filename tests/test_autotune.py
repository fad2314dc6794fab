"""The autotuner's selection rule and bookkeeping on the host (timings injected)."""
import pytest

from paper_2504_14338_gb300 import autotune


def test_pick_fastest_takes_the_minimum_and_the_first_on_ties():
    assert autotune.pick_fastest({1: 5.0, 2: 3.0, 4: 4.0}) == 2
    assert autotune.pick_fastest({4: 2.0, 8: 2.0, 1: 9.0}) == 4
    assert autotune.pick_fastest({8: 1.0}) == 8


def test_injected_timings_drive_the_choice(monkeypatch):
    set_calls = []

    class FakeDp:
        DISCRETE = 0

        @staticmethod
        def dopinf_tune_rollout_rows_large(c):
            set_calls.append(("large", c))
            return 4

        @staticmethod
        def dopinf_tune_rollout_rows(c):
            set_calls.append(("rows", c))
            return 2

        @staticmethod
        def dopinf_tune_reduce_coop(on):
            set_calls.append(("coop", on))
            return 1

    monkeypatch.setattr(autotune, "dp", FakeDp)
    monkeypatch.setattr(autotune, "_key", lambda *a: a)

    class Q:
        shape = (30, 600)

    # r <= 32: rows per CTA of the column-owned rollouts
    small = {1: 9.0, 2: 4.0, 4: 6.5, 8: 7.5}
    out = autotune.tune_learn(Q(), [10, 20, 30], [1] * 8, [1] * 8, 5000, timer=lambda k, c: small[c])
    assert out["best"] == 2 and out["rollout_ms"][2] == 4.0 and set(out["rollout_ms"]) == {1, 2, 4, 8}
    assert out["knob"] == "rollout rows per CTA"
    assert set_calls[-1] == ("rows", 2)  # the winner is set process-wide
    assert len(out["knobs"]) == 1
    # an r above 32 as well: both knobs, the small-r one first
    large = {3: 9.0, 4: 6.0, 5: 4.5, 6: 5.0, 8: 7.0}
    out = autotune.tune_learn(Q(), [10, 40], [1] * 8, [1] * 8, 5000,
                              timer=lambda k, c: large[c] if "> 32" in k else small[c])
    assert out["best"] == 2 and [k["best"] for k in out["knobs"]] == [2, 5]
    assert out["knobs"][1]["rollout_ms"][5] == 4.5
    assert set_calls[-1] == ("large", 5)
    # only r above 32: the large-r knob alone
    out = autotune.tune_learn(Q(), [40, 80], [1] * 8, [1] * 8, 5000, timer=lambda k, c: large[c])
    assert out["best"] == 5 and len(out["knobs"]) == 1
    out = autotune.tune_reduce(Q(), 30, timer={1: 3.0, 0: 7.0}.get)
    assert out["best"] == 1 and set_calls[-1] == ("coop", 1)
