"""Host logic of the launch-parameter autotuner (no GPU: the timer is a fake)."""
import math

import numpy as np
import pytest

from paper_1704_00131_gb300 import autotune as AT
from paper_1704_00131_gb300 import workloads as W


def test_candidates_cover_the_family():
    c = AT.candidates("mixed", (8, 16))
    assert c == [("mixed", 8), ("mixed", 16), ("mixed_tc", 8), ("mixed_tc", 16)]
    assert AT.candidates("fp64", (16,)) == [("fp64", 16)]
    with pytest.raises(ValueError):
        AT.candidates("fp16")
    with pytest.raises(ValueError):
        AT.candidates("mixed", (0,))


def test_choose_fastest_skips_failed_and_keeps_first_on_ties():
    t = [("mixed", 8, 5.0), ("mixed", 16, 3.0), ("mixed_tc", 16, 3.0), ("mixed", 32, math.nan)]
    assert AT.choose(t) == ("mixed", 16, {}, 3.0)
    t2 = [("mixed", 16, {}, 3.0), ("mixed", 16, {"dd_tile": 3}, 2.0)]
    assert AT.choose(t2) == ("mixed", 16, {"dd_tile": 3}, 2.0)
    with pytest.raises(RuntimeError):
        AT.choose([("mixed", 8, math.inf)])


def test_option_candidates():
    assert AT.option_candidates("fp64") == []
    assert AT.option_candidates("mixed") == [{"dd_tile": 3}, {"dd_tile": 4}]
    tc = AT.option_candidates("mixed_tc")
    assert {"tc_min_sites": 1} in tc and {"dd_tile": 4} in tc


def test_signature_depends_on_shapes_not_couplings():
    a = W.config_c3(8)
    b = W.config_c3(8)
    for m in b.models:
        m.U = m.U + 1.0
    ka = AT.signature(a.models, a.chain_model, "mixed", (8, 16))
    assert ka == AT.signature(b.models, b.chain_model, "mixed", (8, 16))
    assert ka != AT.signature(a.models, a.chain_model, "fp64", (8, 16))
    assert ka != AT.signature(a.models, a.chain_model, "mixed", (8, 32))
    c = W.config_c3(16)
    assert ka != AT.signature(c.models, c.chain_model, "mixed", (8, 16))


def test_tune_picks_minimum_and_uses_cache(tmp_path):
    wl = W.config_c3(4)
    calls = []

    def fake(models, cm, p, k, seed, stream, **opt):
        calls.append((p, k, tuple(sorted(opt.items()))))
        base = {("mixed", 8): 7.0, ("mixed", 16): 4.0, ("mixed_tc", 8): 9.0, ("mixed_tc", 16): 6.0}[(p, k)]
        return base - (0.5 if opt.get("dd_tile") == 3 else 0.0)

    cache = AT.Cache(str(tmp_path / "at.json"))
    ch = AT.tune(wl.models, wl.chain_model, "mixed", (8, 16), cache=cache, timer=fake, device="fake-gpu")
    # first pass: family x rank; second pass: the winner's launch options
    assert (ch.precision, ch.delay_k, ch.ms, ch.cached, ch.options) == ("mixed", 16, 3.5, False, {"dd_tile": 3})
    assert len(calls) == 6 and len(ch.timings) == 6
    again = AT.tune(wl.models, wl.chain_model, "mixed", (8, 16), cache=cache, timer=fake, device="fake-gpu")
    assert again.cached and (again.precision, again.delay_k, again.options) == ("mixed", 16, {"dd_tile": 3})
    assert len(calls) == 6
    # another device is tuned afresh
    AT.tune(wl.models, wl.chain_model, "mixed", (8, 16), cache=cache, timer=fake, device="other-gpu")
    assert len(calls) == 12
    # no cache: always tuned
    AT.tune(wl.models, wl.chain_model, "fp64", (8,), cache=None,
            timer=lambda *a, **k: 1.0, device="fake-gpu")


def test_cache_survives_a_corrupt_file(tmp_path):
    p = tmp_path / "at.json"
    p.write_text("{not json")
    cache = AT.Cache(str(p))
    assert cache.get("d", "k") is None
    cache.put("d", "k", AT.Choice("fp64", 16, 1.0, [("fp64", 16, {}, 1.0)]))
    assert cache.get("d", "k").delay_k == 16
