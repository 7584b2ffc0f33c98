"""The oracle against its stored outputs (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone): any change of its
arithmetic shows up here and must be justified by a passage of the paper."""
import importlib.util
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _read(name):
    vals = {}
    with open(os.path.join(HERE, "golden", f"oracle_{name}.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            key, i, v = line.split()
            vals.setdefault(key, {})[int(i)] = float(v)
    return {k: np.array([d[i] for i in range(len(d))]) for k, d in vals.items()}


@pytest.mark.parametrize("name", ["parallel", "cone", "pet"])
def test_oracle_reproduces_stored_outputs(oracle, name):
    from paper_2602_01057_gb300 import synth
    m = _maker()
    (_, gd, G, _), = [c for c in m.cases() if c[0] == name]
    want = _read(name)
    fwd = oracle.forward(gd, G)
    np.testing.assert_allclose(fwd["I"], want["I"], rtol=1e-13, atol=1e-15)
    assert np.count_nonzero(want["I"]) > 10
    bwd = oracle.backward(gd, G, synth.random_weights(synth.num_rays(gd), 7))
    for k in ("mu", "ls", "q", "rho"):
        np.testing.assert_allclose(np.asarray(bwd[k]).reshape(-1), want[f"g_{k}"], rtol=1e-11,
                                   atol=1e-13 * np.abs(want[f"g_{k}"]).max())
