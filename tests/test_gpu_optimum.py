"""The regularised GPU fit against its closed-form optimum.

Constant true maps seen without noise through spatially varying B1 fields
make NLL = 0 and JTV_eps = sum_n sqrt(0 + eps^2) = N eps, both minimal at the
truth (Eqs. 38-40). From a randomly perturbed start, the fit must therefore
return to the truth with F = N eps, and F can never fall below N eps. The
property holds at any size, so it is checked at the benchmark's full size as
well as on a grid with ragged tiles. The noise-free images come from the
oracle's forward model, so the check covers the GPU's signal model too.
"""
import numpy as np
import pytest

import oracle as orc
from cases import f32, round_protocol, to_dev, to_np
from paper_2102_01604_gb300 import phantom

pytestmark = pytest.mark.gpu

EPS = 1e-3


@pytest.fixture(scope="module")
def mpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2102_01604_gb300 as m
    m._lib.load()
    return m


@pytest.mark.parametrize("shape", [(37, 29, 18), (176, 240, 256)])
def test_fit_returns_to_constant_truth(mpm, shape):
    N = int(np.prod(shape))
    prot = round_protocol(phantom.protocol())
    ph = phantom.phantom(shape, seed=2)
    truth = np.tile(ph["y"][:, :1], (1, N))
    b1p, b1m = f32(ph["b1p"]), f32(ph["b1m"])
    s = orc.forward(orc.make_problem(prot, shape), truth, b1p, b1m)
    prot["sigma2"] = [float(np.float32(v)) for v in phantom.noise_sigma2(s, prot)]
    del ph
    problem = mpm.make_problem(prot, shape, lam=10.0, eps=EPS)
    opts = mpm.make_opts(gn_iters=60, cg_iters=30, init=False)
    y0 = truth + np.random.default_rng(7).uniform(-0.1, 0.1, truth.shape)
    y = to_dev(f32(y0))
    st, rep = mpm.mpm_fit(problem, opts, to_dev(f32(s)), y, to_dev(b1p), to_dev(b1m))
    assert rep.iters == 60
    F = np.array(rep.F[:61]) / (N * EPS)
    assert F[0] > 100.0                      # the start is far from the optimum
    assert F[-1] >= 1.0 - 1e-6, F[-1]        # never below N eps
    assert F[-1] <= 1.0 + 1e-3, F[-1]        # and at it
    err = np.abs(to_np(y) - truth) / np.maximum(1.0, np.abs(truth))
    assert err.max() < 1e-3, err.max(axis=1)
