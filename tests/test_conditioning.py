"""Conditioning of the mirror descent (oracle only, CPU): how far the FP64
oracle's GW value moves when every step's cost Pi is perturbed by float32
rounding (relative 6e-8 per entry), the smallest perturbation any float
implementation makes.  Where this exceeds the 1e-5 value bound, a float
solve cannot be held to it; the GPU parity tests choose eps so that it does
not.  The perturbation is the only difference between the two runs."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2404_08970_gb300 import inputs as I


def value_sensitivity(DX, DY, u, v, eps, n_outer, n_inner, rel, seeds=3):
    def run(seed):
        rng = np.random.default_rng(seed)
        T = np.outer(u, v)
        for _ in range(n_outer):
            Pi = 2.0 * O.grad(DX, DY, T, u, v)
            if rel:
                Pi = Pi * (1.0 + rel * rng.uniform(-1.0, 1.0, size=Pi.shape))
            f, g = O.sinkhorn_log(Pi, u, v, eps, n_inner)
            T = O.plan(Pi, f, g, eps)
        return T
    E0 = O.value(DX, DY, run(None))
    return max(abs(O.value(DX, DY, run(s)) - E0) / abs(E0) for s in range(seeds))


def _powk_case(k, eps):
    sx, sy = 9, 12
    rng = I.rng_for(60 + k)
    u, v = I.abs_normal_image(sx, rng), I.abs_normal_image(sy, rng)
    DX = O.grid_dist_2d(sx, 1 / (sx - 1), "manhattan", k)
    DY = O.grid_dist_2d(sy, 1 / (sy - 1), "manhattan", k)
    return DX, DY, u, v


@pytest.mark.parametrize("k,eps,ill", [(2, 5e-2, False), (3, 5e-2, True), (3, 2e-1, False)])
def test_float_rounding_of_pi_moves_the_value(k, eps, ill):
    DX, DY, u, v = _powk_case(k, eps)
    s = value_sensitivity(DX, DY, u, v, eps, 5, 40, 6e-8)
    if ill:
        assert s > 1e-5, s
    else:
        assert s < 2e-6, s
