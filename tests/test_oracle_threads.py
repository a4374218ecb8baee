"""The threaded build of the oracle (OpenMP over voxels, for timing on the
host cores) rounds exactly like the serial build: every volume-wide sum is
taken in the same fixed voxel chunks, so a whole fit, the voxel pass, the prior
and the uncertainty agree bit for bit for any thread count."""
import numpy as np
import pytest

from paper_2102_01604_gb300 import phantom


@pytest.fixture
def threaded(orc):
    yield orc
    orc.use_threads(1)


def _inputs(orc, shape, seed=3):
    prot = phantom.protocol()
    ph = phantom.phantom(shape, seed=seed)
    s = orc.forward(orc.make_problem(prot, shape), ph["y"], ph["b1p"], ph["b1m"])
    prot["sigma2"] = phantom.noise_sigma2(s, prot)
    x = phantom.rician(s, prot, seed=seed + 1)
    return orc.make_problem(prot, shape, lam=10.0, eps=1e-3), x, ph


def _run(orc, p, x, ph):
    fit = orc.fit(p, x, None, ph["b1p"], ph["b1m"], gn_iters=2, cg_iters=10)
    nll, g, h = orc.grad_hess(p, x, fit["y"], ph["b1p"], ph["b1m"])
    e, w = orc.jtv(p, fit["y"])
    var, logdet, mom, st = orc.uncertainty(p, h, w, fit["y"])
    return fit, nll, g, h, e, w, var, logdet, mom, st


@pytest.mark.parametrize("threads", [3, 8])
def test_threaded_oracle_is_bit_identical(threaded, threads):
    orc = threaded
    shape = (40, 32, 12)                      # 15360 voxels: four chunks of 4096
    p, x, ph = _inputs(orc, shape)
    assert orc.use_threads(1) == 1
    ref = _run(orc, p, x, ph)
    assert orc.use_threads(threads) == threads
    got = _run(orc, p, x, ph)
    fr, fg = ref[0], got[0]
    assert fr["iters"] == fg["iters"] == 2
    for k in ("y", "F", "nll", "jtv", "cg_rel"):
        assert np.array_equal(fr[k], fg[k]), k
    for a, b in zip(ref[1:], got[1:]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
