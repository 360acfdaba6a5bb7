"""The autotuner's search space, on the host: it starts from the library's own
defaults (ppsp_options_init), every knob is an option the binding accepts,
and no candidate repeats the default (a wasted trial)."""

import pytest

from paper_2506_16488_gb300 import autotune, ppsp


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()


NAMED = {"strategy": ppsp.STRATEGY, "layout": ppsp.LAYOUT, "frontier": ppsp.FRONTIER}
FIELD = {"strategy": "batch_strategy"}


def test_defaults_are_the_library_defaults():
    o = ppsp.make_options()
    for knob, v in autotune.DEFAULTS.items():
        want = NAMED[knob][v] if knob in NAMED else v
        assert getattr(o, FIELD.get(knob, knob)) == want, knob


def test_every_candidate_is_a_valid_option_and_not_the_default():
    assert {k for k, _ in autotune.SPACE} == set(autotune.DEFAULTS)
    for knob, values in autotune.SPACE:
        assert len(set(values)) == len(values) and autotune.DEFAULTS[knob] not in values, knob
        for v in values:
            kw = {knob: v}
            o = ppsp.make_options(**kw)
            want = NAMED[knob][v] if knob in NAMED else v
            assert getattr(o, FIELD.get(knob, knob)) == want
