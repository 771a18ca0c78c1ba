"""The discrete adjoint (pic_adjoint) against central finite differences,
h = 1e-4, of the FP64 GPU forward run and of the FP64 oracle run, for the
gradient of the beam loss with respect to the laser amplitude a0, the spin
angle of the initial spins and the knots of a piecewise-linear density
profile (through torch autograd), and per particle."""
import math

import numpy as np
import pytest

import oracle
import paper_2002_02211_gb300 as pic
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2002_02211_gb300.autograd import LossRun, PolarizationLoss, forward_loss  # noqa: E402

H = 1e-4
LOSS = dict(axis=1, e_cut_mev=0.25, e_width_mev=0.15)
NSTEPS, K = 26, 7


def _case():
    wl = W.small_case(nx=40, ny=16, ppc=3, a0=2.0, u_th=0.05, seed=31)
    parts = W.generate_particles(wl)
    for k in ("ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz", "w"):
        parts[0][k] = parts[0][k].astype(np.float64)
    x = parts[0]["ix"] + parts[0]["ox"]
    xk = np.linspace(2.0, wl.nx - 2.0, 6)
    return wl, parts, x, xk


def _weights(knots, x, xk, ppc):
    # piecewise-linear density profile through the knots, weight = n(x) / ppc
    i = np.clip(np.searchsorted(xk, x) - 1, 0, len(xk) - 2)
    t = (x - xk[i]) / (xk[i + 1] - xk[i])
    return (knots[i] * (1 - t) + knots[i + 1] * t) / ppc


def _spins(theta, n):
    return np.stack([np.full(n, math.cos(theta)), np.full(n, math.sin(theta)), np.zeros(n)], axis=1)


def _run(wl, parts):
    return LossRun(lambda a0: pic.config_from_workload(W.scaled(wl, a0=a0), precision=64), parts, 0, NSTEPS, K,
                   LOSS, neutralize=False)


def _oracle_loss(wl, parts, a0, w, spins):
    d = dict(parts[0])
    d["w"] = w
    d["sx"], d["sy"], d["sz"] = spins[:, 0], spins[:, 1], spins[:, 2]
    o = oracle.OracleSim(W.scaled(wl, a0=a0), [d])
    o.step(NSTEPS)
    return o.loss(0, **LOSS)


def test_adjoint_gradient_matches_finite_differences_of_gpu_and_oracle():
    wl, parts, x, xk = _case()
    n = len(x)
    run = _run(wl, parts)
    knots0 = np.array([0.03, 0.05, 0.06, 0.05, 0.04, 0.05])
    theta0, a00 = 1.3, 2.0
    # adjoint through torch: parameters -> (weights, spins) -> loss
    a0 = torch.tensor(a00, dtype=torch.float64, requires_grad=True)
    knots = torch.tensor(knots0, dtype=torch.float64, requires_grad=True)
    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    xt, xkt = torch.from_numpy(x), torch.from_numpy(xk)
    i = torch.clamp(torch.searchsorted(xkt, xt) - 1, 0, len(xk) - 2)
    t = (xt - xkt[i]) / (xkt[i + 1] - xkt[i])
    w = (knots[i] * (1 - t) + knots[i + 1] * t) / wl.species[0].ppc
    spins = torch.stack([torch.cos(theta).expand(n), torch.sin(theta).expand(n), torch.zeros(n, dtype=torch.float64)],
                        dim=1)
    L = PolarizationLoss(a0, w, spins, run)
    L.backward()
    grads = {"a0": a0.grad.item(), "theta": theta.grad.item(), "k1": knots.grad[1].item(),
             "k4": knots.grad[4].item()}
    # the loss value agrees with the oracle's
    w0 = _weights(knots0, x, xk, wl.species[0].ppc)
    assert L.item() == pytest.approx(_oracle_loss(wl, parts, a00, w0, _spins(theta0, n)), rel=1e-9, abs=1e-12)

    def evals(f):
        out = {}
        for key in grads:
            vals = []
            for sgn in (1, -1):
                a, th, kn = a00, theta0, knots0.copy()
                if key == "a0":
                    a += sgn * H
                elif key == "theta":
                    th += sgn * H
                else:
                    kn[int(key[1])] += sgn * H
                vals.append(f(a, _weights(kn, x, xk, wl.species[0].ppc), _spins(th, n)))
            out[key] = (vals[0] - vals[1]) / (2 * H)
        return out

    fd_gpu = evals(lambda a, ww, ss: forward_loss(run, a, ww, ss))
    fd_orc = evals(lambda a, ww, ss: _oracle_loss(wl, parts, a, ww, ss))
    scale = max(abs(v) for v in grads.values())
    for key, g in grads.items():
        for name, fd in (("gpu", fd_gpu[key]), ("oracle", fd_orc[key])):
            assert abs(g - fd) <= 1e-3 * max(abs(fd), 1e-2 * scale), (key, name, g, fd, grads, fd_gpu, fd_orc)
    assert abs(grads["a0"]) > 0 and abs(grads["theta"]) > 0


def test_per_particle_gradients_match_finite_differences():
    # one particle's perturbation can move a cell crossing across a step (the
    # Esirkepov current is continuous but its slope jumps there), which a
    # difference step of 1e-4 straddles; 1e-6 stays on one side (FP64 keeps
    # the quotient at 1e-9 relative)
    h = 1e-6
    wl, parts, x, xk = _case()
    run = _run(wl, parts)
    w0 = parts[0]["w"].copy()
    spins0 = np.stack([parts[0]["sx"], parts[0]["sy"], parts[0]["sz"]], axis=1)
    with run.start(2.0, w0, spins0) as sim:
        sim.adjoint(NSTEPS, K, species=0, **LOSS)
        g = sim.adjoint_particle_grads(0)
    order = np.argsort(g["id"])
    # the particles with the largest momentum gradient
    pick = order[np.argsort(-np.abs(g["ux"][order]))[:2]]
    for slot in pick:
        pid = g["id"][slot]
        for key in ("ux", "ox", "sy", "w"):
            vals = []
            for sgn in (1, -1):
                p2 = [dict(parts[0])]
                arr = p2[0][key].astype(np.float64).copy()
                arr[pid] += sgn * h
                p2[0][key] = arr
                r2 = _run(wl, p2)
                vals.append(forward_loss(r2, 2.0, p2[0]["w"], np.stack([p2[0]["sx"], p2[0]["sy"], p2[0]["sz"]], 1)))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(g[key][slot] - fd) <= 1e-4 * abs(fd) + 1e-9, (pid, key, g[key][slot], fd)


def test_fp32_adjoint_matches_fp64_adjoint_and_finite_differences():
    # the FP32 adjoint (the one the benchmark times) differentiates the FP32
    # forward run; it follows the FP64 adjoint, and the FP64 central
    # differences, within the 1e-3 relative bar of the FP64 check (FP32
    # rounding of the forward states moves the gradient by about 1e-6 here)
    wl, parts, x, xk = _case()
    n = len(x)
    knots0 = np.array([0.03, 0.05, 0.06, 0.05, 0.04, 0.05])
    w0 = _weights(knots0, x, xk, wl.species[0].ppc)
    theta0, a00 = 1.3, 2.0
    grads = {}
    for prec in (32, 64):
        run = LossRun(lambda a0, p=prec: pic.config_from_workload(W.scaled(wl, a0=a0), precision=p), parts, 0,
                      NSTEPS, K, LOSS, neutralize=False)
        with run.start(a00, w0, _spins(theta0, n)) as sim:
            L, dla0 = sim.adjoint(NSTEPS, K, species=0, **LOSS)
            g = sim.adjoint_particle_grads(0)
        gw, gs = np.zeros(n), np.zeros((n, 3))
        gw[g["id"]] = g["w"]
        gs[g["id"], 0], gs[g["id"], 1] = g["sx"], g["sy"]
        grads[prec] = {"L": L, "a0": dla0,
                       "theta": float(np.sum(-math.sin(theta0) * gs[:, 0] + math.cos(theta0) * gs[:, 1])),
                       "w_norm": float(np.linalg.norm(gw))}
    run64 = _run(wl, parts)
    fd = {}
    for key in ("a0", "theta"):
        vals = []
        for sgn in (1, -1):
            a, th = a00 + (sgn * H if key == "a0" else 0.0), theta0 + (sgn * H if key == "theta" else 0.0)
            vals.append(forward_loss(run64, a, w0, _spins(th, n)))
        fd[key] = (vals[0] - vals[1]) / (2 * H)
    assert grads[32]["L"] == pytest.approx(grads[64]["L"], rel=1e-5)
    for key in ("a0", "theta", "w_norm"):
        assert grads[32][key] == pytest.approx(grads[64][key], rel=1e-3), (key, grads)
    for key in ("a0", "theta"):
        assert abs(grads[32][key] - fd[key]) <= 1e-3 * abs(fd[key]), (key, grads[32][key], fd[key])
