"""The stored expected values under tests/golden/ are the ones the committed generator writes from the
oracle (no hand-edited numbers)."""
import importlib.util
import json
import os

import numpy as np


def test_ghat_quadrature_golden_is_what_the_generator_writes(repo_root):
    gdir = os.path.join(repo_root, "tests", "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(gdir, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    fresh = mod.ghat_quadrature()
    with open(os.path.join(gdir, "ghat_t_quadrature.json")) as fh:
        stored = json.load(fh)
    assert stored["source"] == fresh["source"]
    for key in ("kb", "R"):
        assert np.isclose(stored[key], fresh[key], rtol=1e-14, atol=0)
    np.testing.assert_allclose(stored["w"], fresh["w"], rtol=1e-14, atol=0)
    got = np.array(fresh["re"]) + 1j * np.array(fresh["im"])
    want = np.array(stored["re"]) + 1j * np.array(stored["im"])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
