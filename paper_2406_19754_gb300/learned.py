"""Learned l1-Jacobi damping weights: binding, training loop and evaluation.

The network (include/amg.h, mlp_*) maps nine stencil features of each row to
omega_i in (0, omega_max] (omega_max 1 by default, or up to below 2, which
still keeps the smoother A-convergent); the smoother scale becomes
s_i = omega_i / d_i.  Training
minimises the two-grid error-reduction loss (amg_twogrid_loss) over
generated variable-coefficient diffusion problems with Adam.  Every numeric
step runs in the library's kernels; this module only sequences the calls.

  python -m paper_2406_19754_gb300.learned train --problems 4000 [--omega-max 1.9]
  python -m paper_2406_19754_gb300.learned evaluate [--omega-max 1.9] [--weights FILE]
"""

from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import sys
import time

import numpy as np
import torch

from . import Hierarchy, _check, _dev, _ptr, _stream, csr_struct, csr_to_device
from . import _lib

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "omega_mlp_diffusion48.f32")


def weights_path(omega_max: float = 1.0) -> str:
    """The committed network trained with this output cap (1: DEFAULT_WEIGHTS)."""
    if omega_max == 1.0:
        return DEFAULT_WEIGHTS
    return os.path.join(HERE, "weights", "omega_mlp_diffusion48_wmax%g.f32" % omega_max)


class Mlp:
    """The 9 -> 32 -> 32 -> 1 network on the current CUDA device; its output is
    omega = max(omega_max * sigmoid(z), 1e-3) with omega_max in [1, 2)."""

    def __init__(self, seed: int = 0, omega_max: float = 1.0):
        self._lib = _lib.load()
        self.nparam = self._lib.mlp_num_params()
        h = C.c_void_p()
        _check(self._lib.mlp_create(C.c_uint64(seed), C.byref(h)), "mlp_create")
        self.h = h
        self.omega_max = float(omega_max)
        _check(self._lib.mlp_set_omega_max(self.h, self.omega_max), "mlp_set_omega_max")

    def set_exact_forward(self, exact: bool = True) -> None:
        """FP32 CUDA-core forward pass (True) or the tensor-core one (False, default)."""
        _check(self._lib.mlp_set_exact_forward(self.h, 1 if exact else 0),
               "mlp_set_exact_forward")

    def start_at_plain_smoother(self) -> None:
        """Output bias so that a zero hidden signal gives omega = 1 (plain
        l1-Jacobi) under the cap omega_max > 1: sigmoid(b3) = 1 / omega_max."""
        if self.omega_max > 1.0:
            p = self.params()
            p[-1] = np.float32(-np.log(self.omega_max - 1.0))
            self.set_params(p)

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and self.h.value:
                self._lib.mlp_destroy(self.h)
        except Exception:
            pass

    def params(self) -> np.ndarray:
        p = np.empty(self.nparam, dtype=np.float32)
        _check(self._lib.mlp_get_params(self.h, p.ctypes.data_as(C.c_void_p)))
        return p

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparam
        _check(self._lib.mlp_set_params(self.h, p.ctypes.data_as(C.c_void_p)))

    def grad(self) -> np.ndarray:
        g = np.empty(self.nparam, dtype=np.float64)
        _check(self._lib.mlp_get_grad(self.h, g.ctypes.data_as(C.c_void_p)))
        return g

    def save(self, path: str) -> None:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        self.params().astype("<f4").tofile(path)

    def load(self, path: str) -> None:
        self.set_params(np.fromfile(path, dtype="<f4"))

    def features(self, A, shape, stream=None):
        """A: (rowptr, col, val) CUDA tensors of a 7-point operator on grid (nz, ny, nx)."""
        nz, ny, nx = shape
        Ac, keep = csr_struct(*A)
        feat = torch.empty((Ac.n, 9), dtype=torch.float32, device=keep[0].device)
        _check(self._lib.mlp_features(C.byref(Ac), nx, ny, nz, _ptr(feat), _stream(stream)),
               "mlp_features")
        return feat

    def forward(self, feat, out=None, stream=None):
        feat = _dev(feat, torch.float32, "feat")
        om = out if out is not None else torch.empty(feat.shape[0], dtype=torch.float32,
                                                       device=feat.device)
        _check(self._lib.mlp_forward(self.h, feat.shape[0], _ptr(feat), _ptr(om),
                                     _stream(stream)), "mlp_forward")
        return om

    def backward(self, feat, domega, accumulate=True, stream=None):
        feat = _dev(feat, torch.float32, "feat")
        domega = _dev(domega, torch.float32, "domega")
        _check(self._lib.mlp_backward(self.h, feat.shape[0], _ptr(feat), _ptr(domega),
                                      1 if accumulate else 0, _stream(stream)), "mlp_backward")

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0, stream=None):
        _check(self._lib.mlp_adam_step(self.h, lr, beta1, beta2, eps, grad_scale,
                                       _stream(stream)), "mlp_adam_step")


def twogrid_loss(H: Hierarchy, e0, ncycles=2, gradient=True, stream=None):
    """(loss, d loss / d omega) of the weights set on H; e0: (nsamples, n) float64."""
    e0 = _dev(e0, torch.float64, "e0")
    lib = _lib.load()
    loss = C.c_double()
    dom = torch.empty(e0.shape[1], dtype=torch.float32, device=e0.device) if gradient else None
    _check(lib.amg_twogrid_loss(H.h, e0.shape[0], ncycles, _ptr(e0), C.byref(loss), _ptr(dom),
                                _stream(stream)), "amg_twogrid_loss")
    return loss.value, dom


# ------------------------------------------------------------------ training

TRAIN_SIDE, TRAIN_ELL, TRAIN_SEED0 = 48, 8.0, 10000
SIGMA_MAX = 3.0
SAMPLES, CYCLES = 4, 2


def training_problem(k: int, side: int = TRAIN_SIDE):
    """Problem k: diffusion on side^3 with k = exp(g), sigma ~ U[0, 3] (seeded)."""
    from synthetic import diffusion_problem, standard_normal, uniform01

    seed = TRAIN_SEED0 + k
    sigma = float(uniform01(seed, 1)[0]) * SIGMA_MAX
    A = diffusion_problem(side, sigma, TRAIN_ELL, seed)
    n = side ** 3
    e0 = standard_normal(seed + 7919, SAMPLES * n).reshape(SAMPLES, n)
    return A, e0, sigma


def _load_problem(args):
    k, side = args
    A, e0, sigma = training_problem(k, side)
    return k, A, e0, sigma


def train(mlp: Mlp, problems: int, batch: int = 8, lr: float = 1e-3, side: int = TRAIN_SIDE,
          workers: int = 4, log=None):
    """One epoch over `problems` generated problems, Adam step every `batch`."""
    import concurrent.futures as cf
    import multiprocessing as mp

    dev = torch.device("cuda")
    hist = []
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        it = ex.map(_load_problem, [(k, side) for k in range(problems)], chunksize=2)
        t0 = time.time()
        for k, A, e0, sigma in it:
            Ad = csr_to_device(A, dev)
            H = Hierarchy(*Ad)
            feat = mlp.features(Ad, (side, side, side))
            om = mlp.forward(feat)
            H.set_smoother_weights(om)
            loss, dom = twogrid_loss(H, torch.as_tensor(e0, device=dev), CYCLES)
            mlp.backward(feat, dom, accumulate=(k % batch) != 0)
            H.close()
            hist.append((k, sigma, loss))
            if (k + 1) % batch == 0 or k + 1 == problems:
                mlp.adam(lr=lr, grad_scale=1.0 / batch)
            if log and (k + 1) % 100 == 0:
                recent = [h[2] for h in hist[-100:]]
                log("%5d problems  mean loss (last 100) %.5f  %.1f s" %
                    (k + 1, float(np.mean(recent)), time.time() - t0))
    return hist


def evaluate(weights: str | None, side: int = 256, sigma: float = 2.5, seed: int = 5,
             precision: str = "f64", tol: float = 1e-8, repeats: int = 3,
             omega_max: float = 1.0):
    """Iterations and seconds to tol on side^3 diffusion: omega == 1 (plain
    l1-Jacobi), the network, and the constant omega equal to the network's
    mean (does the per-row choice matter, or only the overall step?)."""
    from synthetic import diffusion_problem, uniform01

    dev = torch.device("cuda")
    A = diffusion_problem(side, sigma, TRAIN_ELL, seed)
    Ad = csr_to_device(A, dev)
    b = torch.as_tensor(uniform01(seed + 1, side ** 3), device=dev)
    H = Hierarchy(*Ad, precision=precision)

    def timed():
        best, info = None, None
        for _ in range(repeats):
            x = torch.zeros_like(b)
            _, info = H.pcg(b, x, tol=tol)
            best = info["solve_ms"] if best is None else min(best, info["solve_ms"])
        return info["iterations"], best / 1e3, info["true_relres"]

    out = {"side": side, "sigma": sigma, "seed": seed, "precision": precision, "tol": tol}
    out["plain"] = dict(zip(("iterations", "seconds", "true_relres"), timed()))
    mlp = Mlp(0, omega_max)
    if weights:
        mlp.load(weights)
    feat = mlp.features(Ad, (side, side, side))
    om = mlp.forward(feat)
    # inference cost per evaluation: features + forward + new smoother scales
    def ms(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeats):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / repeats

    def infer():
        mlp.forward(mlp.features(Ad, (side, side, side)), out=om)
        H.set_smoother_weights(om)

    out["inference_ms"] = ms(infer)
    out["features_ms"] = ms(lambda: mlp.features(Ad, (side, side, side)))
    out["set_weights_ms"] = ms(lambda: H.set_smoother_weights(om))
    fw0, fw1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fw0.record()
    for _ in range(repeats):
        mlp.forward(feat, out=om)
    fw1.record()
    torch.cuda.synchronize()
    out["forward_ms"] = fw0.elapsed_time(fw1) / repeats
    H.set_smoother_weights(om)
    out["learned"] = dict(zip(("iterations", "seconds", "true_relres"), timed()))
    out["omega_mean"] = float(om.mean())
    out["omega_min"] = float(om.min())
    out["omega_max"] = float(om.max())
    out["omega_cap"] = omega_max
    H.set_smoother_weights(torch.full_like(om, float(om.mean())))
    out["constant_mean_omega"] = dict(zip(("iterations", "seconds", "true_relres"), timed()))
    H.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--problems", type=int, default=4000)
    t.add_argument("--batch", type=int, default=8)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--side", type=int, default=TRAIN_SIDE)
    t.add_argument("--seed", type=int, default=0)
    t.add_argument("--workers", type=int, default=8)
    t.add_argument("--omega-max", type=float, default=1.0,
                   help="output cap in [1, 2): omega = max(cap * sigmoid(z), 1e-3)")
    t.add_argument("--out", default=None)
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", default=None)
    e.add_argument("--omega-max", type=float, default=1.0)
    e.add_argument("--side", type=int, default=256)
    e.add_argument("--sigma", type=float, default=2.5)
    e.add_argument("--precision", default="f64")
    a = ap.parse_args(argv)
    if a.cmd == "train":
        a.out = a.out or weights_path(a.omega_max)
        mlp = Mlp(a.seed, a.omega_max)
        mlp.start_at_plain_smoother()
        hist = train(mlp, a.problems, a.batch, a.lr, a.side, a.workers,
                     log=lambda s: print(s, flush=True))
        mlp.save(a.out)
        first = float(np.mean([h[2] for h in hist[:100]]))
        last = float(np.mean([h[2] for h in hist[-100:]]))
        print(json.dumps({"problems": a.problems, "loss_first100": first,
                          "loss_last100": last, "weights": a.out}), flush=True)
    else:
        print(json.dumps(evaluate(a.weights or weights_path(a.omega_max), a.side, a.sigma,
                                  precision=a.precision, omega_max=a.omega_max)), flush=True)


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(HERE))
    main()
