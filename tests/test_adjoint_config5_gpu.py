"""The adjoint at the scale of the gradient study: 1024 x 512 cells, 8
electrons per cell (4.18 million) whose density follows the 64-knot ramp,
laser a0 = 5, loss the energy-weighted polarization s_y above 50 MeV (width
5 MeV), checkpoints every 50 steps.

The horizon is 200 steps, the longest at which an h = 1e-4 central
difference still measures the derivative of the discrete run: there the
h = 1e-4 and h = 1e-6 differences of dL/da0 agree to about 1e-4 (at 250
steps they part by 1e-3, and further on the run's sensitivity to a0 grows
until no difference of that size follows the derivative).  Checked: the FP64
adjoint's dL/da0, dL/d(spin angle) and dL/d(two ramp knots) against h = 1e-4
central differences of the FP64 forward path within 1e-3, and the FP32
adjoint against the FP64 one within 1e-3.
"""
import math

import numpy as np
import pytest

import paper_2002_02211_gb300 as pic
import workloads as W

pytestmark = pytest.mark.gpu
pytest.importorskip("torch")
from paper_2002_02211_gb300.autograd import LossRun, forward_loss  # noqa: E402

HORIZON, K, H = 200, 50, 1e-4
LOSS = dict(axis=1, e_cut_mev=50.0, e_width_mev=5.0)
KNOTS = (16, 40)


def test_config5_adjoint_against_finite_differences_and_fp32():
    wl = W.CONFIG5
    parts = W.generate_particles(wl)
    for k in ("ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz", "w"):
        parts[0][k] = parts[0][k].astype(np.float64)
    x = parts[0]["ix"] + parts[0]["ox"]
    knots0 = W.ramp_knots()
    xk = np.linspace(2.0, wl.nx - 2.0, len(knots0))
    i = np.clip(np.searchsorted(xk, x) - 1, 0, len(xk) - 2)
    t = (x - xk[i]) / (xk[i + 1] - xk[i])
    ppc = wl.species[0].ppc
    n = len(x)

    def weights(kn):
        return (kn[i] * (1 - t) + kn[i + 1] * t) / ppc

    def spins(th):
        return np.stack([np.full(n, math.cos(th)), np.full(n, math.sin(th)), np.zeros(n)], 1)

    theta0, a00 = math.pi / 2, wl.a0
    runs = {p: LossRun(lambda a0, p=p: pic.config_from_workload(W.scaled(wl, a0=a0), precision=p), parts, 0,
                       HORIZON, K, LOSS, neutralize=True) for p in (32, 64)}
    grads = {}
    for prec, run in runs.items():
        with run.start(a00, weights(knots0), spins(theta0)) as sim:
            _, dla0 = sim.adjoint(HORIZON, K, species=0, **LOSS)
            g = sim.adjoint_particle_grads(0)
        gw, gsx, gsy = np.zeros(n), np.zeros(n), np.zeros(n)
        gw[g["id"]], gsx[g["id"]], gsy[g["id"]] = g["w"], g["sx"], g["sy"]
        d = {"a0": dla0, "theta": float(np.sum(-math.sin(theta0) * gsx + math.cos(theta0) * gsy))}
        for j in KNOTS:   # the weights are linear in the knots
            d[f"k{j}"] = float(np.sum(gw * ((i == j) * (1 - t) + (i + 1 == j) * t) / ppc))
        grads[prec] = d
    for key, g in grads[64].items():
        vals = []
        for sgn in (1, -1):
            a, th, kn = a00, theta0, knots0.copy()
            if key == "a0":
                a += sgn * H
            elif key == "theta":
                th += sgn * H
            else:
                kn[int(key[1:])] += sgn * H
            vals.append(forward_loss(runs[64], a, weights(kn), spins(th)))
        fd = (vals[0] - vals[1]) / (2 * H)
        assert g != 0.0
        assert abs(g - fd) <= 1e-3 * abs(fd), (key, g, fd)
        assert abs(grads[32][key] - g) <= 1e-3 * abs(g), (key, grads[32][key], g)
