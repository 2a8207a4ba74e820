"""Amortised FSI explainer: a student network trained on exact FSI.

The student maps an instance x straight to its FSI scores, skipping the 2^d
masked-model evaluations and the exact transform.  Its training pairs
(x, FSI(v_x)) come from the exact path of this library (the masked-game
kernel for v_x, then tt_fsi_apply); its forward and backward passes run on
the tcgen05 BF16 GEMM with FP32 accumulation and a fused Adam step; its
outputs are projected onto the efficiency constraint.  At inference a
residual spot check on sampled coalitions compares the student's order-l
surrogate with the model's values; instances that fail it are recomputed on
the exact path.

This module sequences calls into the C ABI (include/tt_fsi.h); every
arithmetic step runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import math
import struct
from dataclasses import dataclass

import numpy as np

from . import (ARITH, DeviceMLP, FsiError, Plan, _check, _stream_ptr, masked_game_into, masked_game_tc, native,
               num_scores, score_masks)
from . import synthetic

_SIGS_DONE = False


def _declare():
    global _SIGS_DONE
    if _SIGS_DONE:
        return native.load()
    lib = native.load()
    c = ctypes
    i, i64, vp, f = c.c_int, c.c_int64, c.c_void_p, c.c_float
    lib.tt_fsi_student_create.restype = i
    lib.tt_fsi_student_create.argtypes = [i, i, i, i, vp, c.POINTER(vp)]
    lib.tt_fsi_student_destroy.restype = None
    lib.tt_fsi_student_destroy.argtypes = [vp]
    lib.tt_fsi_student_num_params.restype = i64
    lib.tt_fsi_student_num_params.argtypes = [vp]
    lib.tt_fsi_student_set_adam.restype = i
    lib.tt_fsi_student_set_adam.argtypes = [vp, f, f, f, f]
    for name in ("tt_fsi_student_gradients", "tt_fsi_student_train_step"):
        getattr(lib, name).restype = i
        getattr(lib, name).argtypes = [vp, vp, vp, vp, f, i, vp, vp]
    lib.tt_fsi_student_predict.restype = i
    lib.tt_fsi_student_predict.argtypes = [vp, vp, vp, f, i, vp, vp]
    lib.tt_fsi_student_get_state.restype = i
    lib.tt_fsi_student_get_state.argtypes = [vp, vp, vp, vp, c.POINTER(i64)]
    lib.tt_fsi_student_set_state.restype = i
    lib.tt_fsi_student_set_state.argtypes = [vp, vp, vp, vp, i64]
    lib.tt_fsi_student_get_grads.restype = i
    lib.tt_fsi_student_get_grads.argtypes = [vp, vp]
    lib.tt_fsi_student_check.restype = i
    lib.tt_fsi_student_check.argtypes = [vp, vp]
    lib.tt_fsi_surrogate_residual.restype = i
    lib.tt_fsi_surrogate_residual.argtypes = [vp, i, i, vp, vp, vp, i, vp, vp]
    lib.tt_fsi_masked_game_sampled.restype = i
    lib.tt_fsi_masked_game_sampled.argtypes = [vp, vp, vp, i64, vp, i, vp, vp]
    _SIGS_DONE = True
    return lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def init_params(d: int, hidden: int, n_out: int, seed: int, out_scale: float = 0.01) -> np.ndarray:
    """Weights N(0, 1/fan_in), zero biases, drawn from the seeded stream; the
    output layer is further scaled by out_scale so that the first outputs
    are small next to the FSI scores (faster, steadier training)."""
    st = synthetic.Stream(seed, synthetic.TAG_STUDENT)
    W1 = st.normal(hidden * d) / math.sqrt(d)
    W2 = st.normal(hidden * hidden) / math.sqrt(hidden)
    W3 = st.normal(n_out * hidden) / math.sqrt(hidden) * out_scale
    return np.concatenate([W1, np.zeros(hidden), W2, np.zeros(hidden), W3, np.zeros(n_out)]).astype(np.float32)


class Student:
    """The student network on the GPU (C ABI handle)."""

    def __init__(self, d: int, hidden: int, n_out: int, max_batch: int, params: np.ndarray):
        self._lib = _declare()
        self.d, self.hidden, self.n_out, self.max_batch = d, hidden, n_out, max_batch
        p = np.ascontiguousarray(params, dtype=np.float32)
        h = ctypes.c_void_p()
        _check(self._lib.tt_fsi_student_create(d, hidden, n_out, max_batch, p.ctypes.data, ctypes.byref(h)),
               "tt_fsi_student_create")
        self._h = h
        self.n_params = int(self._lib.tt_fsi_student_num_params(h))
        import torch
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tt_fsi_student_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(self._lib.tt_fsi_student_set_adam(self._h, lr, beta1, beta2, eps), "tt_fsi_student_set_adam")

    def gradients(self, x, labels, target, v_empty: float):
        _check(self._lib.tt_fsi_student_gradients(self._h, _p(x), _p(labels), _p(target), v_empty, x.shape[0],
                                                  _p(self._loss), _stream_ptr()), "tt_fsi_student_gradients")
        return self._loss

    def train_step(self, x, labels, target, v_empty: float):
        """One forward/backward/Adam step; returns the loss as a device scalar."""
        _check(self._lib.tt_fsi_student_train_step(self._h, _p(x), _p(labels), _p(target), v_empty, x.shape[0],
                                                   _p(self._loss), _stream_ptr()), "tt_fsi_student_train_step")
        return self._loss

    def predict(self, x, target, v_empty: float, out=None):
        import torch
        if out is None:
            out = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=x.device)
        _check(self._lib.tt_fsi_student_predict(self._h, _p(x), _p(target), v_empty, x.shape[0], _p(out),
                                                _stream_ptr()), "tt_fsi_student_predict")
        return out

    def check(self):
        _check(self._lib.tt_fsi_student_check(self._h, _stream_ptr()), "tt_fsi_student_check")

    def grads(self) -> np.ndarray:
        g = np.empty(self.n_params, dtype=np.float32)
        _check(self._lib.tt_fsi_student_get_grads(self._h, g.ctypes.data), "tt_fsi_student_get_grads")
        return g

    def state(self):
        p = np.empty(self.n_params, dtype=np.float32)
        m = np.empty_like(p)
        v = np.empty_like(p)
        step = ctypes.c_int64()
        _check(self._lib.tt_fsi_student_get_state(self._h, p.ctypes.data, m.ctypes.data, v.ctypes.data,
                                                  ctypes.byref(step)), "tt_fsi_student_get_state")
        return p, m, v, int(step.value)

    def load_state(self, p, m, v, step: int):
        p, m, v = (np.ascontiguousarray(a, dtype=np.float32) for a in (p, m, v))
        _check(self._lib.tt_fsi_student_set_state(self._h, p.ctypes.data, m.ctypes.data, v.ctypes.data, step),
               "tt_fsi_student_set_state")

    # checkpoint file: magic, version, d, hidden, n_out, step, then params, m, v
    _MAGIC = b"TTFSISTU"

    def save(self, path: str):
        p, m, v, step = self.state()
        with open(path, "wb") as f:
            f.write(self._MAGIC + struct.pack("<iiiiq", 1, self.d, self.hidden, self.n_out, step))
            for a in (p, m, v):
                f.write(a.astype("<f4").tobytes())

    def load(self, path: str):
        with open(path, "rb") as f:
            head = f.read(8 + 24)
            if head[:8] != self._MAGIC:
                raise ValueError("not a student checkpoint")
            ver, d, hidden, n_out, step = struct.unpack("<iiiiq", head[8:])
            if (ver, d, hidden, n_out) != (1, self.d, self.hidden, self.n_out):
                raise ValueError("checkpoint does not match this student")
            arrs = [np.frombuffer(f.read(4 * self.n_params), dtype="<f4") for _ in range(3)]
        self.load_state(*arrs, step)


@dataclass
class Dataset:
    x: "object"        # [n, d] float32 (device)
    labels: "object"   # [n, n_out] float32 (device), exact FSI
    target: "object"   # [n] float32 (device), v(N) - v(empty)
    v_empty: float


def sample_coalitions(n: int, d: int, K: int, seed: int, first: int = 0) -> np.ndarray:
    """K coalitions per instance: a size t in 1..d-1 with probability
    proportional to the Shapley kernel (d-1)/(t (d-t)), then a uniform subset
    of that size (a random permutation's first t players).  uint32 masks."""
    st = synthetic.Stream(seed * 1000003 + first, synthetic.TAG_SPOT)
    t = np.arange(1, d)
    w = (d - 1) / (t * (d - t))
    cdf = np.cumsum(w / w.sum())
    u = st.uniform(n * K).reshape(n, K)
    sizes = 1 + np.searchsorted(cdf, u, side="right").clip(max=d - 2)
    keys = st.uniform(n * K * d).reshape(n, K, d)
    order = np.argsort(keys, axis=2)
    ranks = np.argsort(order, axis=2)
    inside = ranks < sizes[:, :, None]
    return (inside * (1 << np.arange(d, dtype=np.uint64))).sum(axis=2).astype(np.uint32)


class Explainer:
    """Teacher model + exact FSI path + student, for one (d, l)."""

    def __init__(self, mlp, ell: int, hidden: int = 1024, batch: int = 4096, seed: int = 4,
                 baseline=None, K: int = 64, value_path: str = "tc"):
        """value_path "tc": the teacher's values for labels, spot checks and the
        fallback of ``explain`` come from the tensor-core kernel (BF16
        layer-2 products, about 0.3 % of max|v|); "f32": from the FP32
        CUDA-core kernels."""
        import torch
        self.torch = torch
        self.mlp = DeviceMLP(mlp, "cuda")
        self.tc = value_path == "tc" and self.mlp.h1 == 128 and self.mlp.h2 == 128 and self.mlp.d >= 7
        self.d, self.ell, self.batch, self.K = self.mlp.d, ell, batch, K
        self.n_out = num_scores(self.d, ell)
        self.baseline = torch.zeros(self.d, dtype=torch.float64, device="cuda") if baseline is None else \
            torch.as_tensor(baseline, dtype=torch.float64, device="cuda")
        self.plan = Plan(self.d, ell, "exact", max_batch=batch)
        self.student = Student(self.d, hidden, self.n_out, batch, init_params(self.d, hidden, self.n_out, seed))
        self.masks = torch.as_tensor(score_masks(self.d, ell).astype(np.uint32).view(np.int32), device="cuda")
        self.v_empty = float(self.values_at(torch.zeros((1, self.d), dtype=torch.float64, device="cuda"),
                                            np.zeros((1, 1), dtype=np.uint32))[0, 0].item())
        self.tau = float("inf")
        self.seed = seed
        # Spot-check coalitions: one pool of `batch` x K draws, made once, so
        # the instance in row i of every call uses pool row i.
        self.coal_pool = sample_coalitions(batch, self.d, K, seed)
        self.coal_pool_dev = torch.as_tensor(self.coal_pool.view(np.int32), device="cuda")

    # -- the exact path -----------------------------------------------------
    def _values_listed(self, x64, c, out, tc):
        if tc:
            return masked_game_tc(self.mlp, x64, self.baseline, coalitions=c, out=out)
        _check(_declare().tt_fsi_masked_game_sampled(ctypes.byref(self.mlp.struct), _p(x64), _p(self.baseline),
                                                      x64.shape[0], _p(c), c.shape[1], _p(out), _stream_ptr()),
               "tt_fsi_masked_game_sampled")
        return out

    def values_at(self, x64, coal: np.ndarray):
        """Teacher values at given coalitions (FP32), [B, K]."""
        torch = self.torch
        c = torch.as_tensor(np.ascontiguousarray(coal, dtype=np.uint32).view(np.int32), device="cuda")
        out = torch.empty(c.shape, dtype=torch.float32, device="cuda")
        return self._values_listed(x64, c, out, self.tc)

    def exact(self, x64, tc=None):
        """FSI of the teacher's masked games by the exact transform (value
        vectors in FP32 from the tensor-core or the CUDA-core kernel, widened
        to FP64)."""
        torch = self.torch
        tc = self.tc if tc is None else tc
        n = x64.shape[0]
        out = torch.empty((n, self.n_out), dtype=torch.float64, device="cuda")
        v32 = torch.empty((min(n, self.batch), 1 << self.d), dtype=torch.float32, device="cuda")
        for s in range(0, n, self.batch):
            e = min(n, s + self.batch)
            vv = v32[:e - s]
            if tc:
                masked_game_tc(self.mlp, x64[s:e], self.baseline, out=vv)
            else:
                masked_game_into(self.mlp, x64[s:e], self.baseline, vv)
            self.plan.apply(vv.double(), out=out[s:e])
        self.plan.check()
        return out

    def targets(self, x64):
        """v(N) - v(empty) for each instance (teacher on the full input)."""
        full = np.full((x64.shape[0], 1), (1 << self.d) - 1, dtype=np.uint32)
        return self.values_at(x64, full)[:, 0] - self.v_empty

    def dataset(self, n: int, first: int = 0, ar1_rho: float = 0.5, seed: int = 4) -> Dataset:
        torch = self.torch
        x = synthetic.gaussian_instances(n, self.d, seed, ar1_rho=ar1_rho, first=first)
        x64 = torch.as_tensor(x, dtype=torch.float64, device="cuda")
        labels = self.exact(x64).float()
        return Dataset(x64.float(), labels, self.targets(x64), self.v_empty)

    # -- training -------------------------------------------------------------
    def train(self, data: Dataset, epochs: int, lr: float = 1e-3, seed: int = 4, log=None,
              schedule: str = "constant"):
        """Adam over the fixed batches of ``data`` for ``epochs`` epochs;
        schedule "cosine" decays the learning rate from lr towards 0 over
        the run (one value per epoch), "constant" keeps it."""
        torch = self.torch
        self.student.set_adam(lr=lr)
        n = data.x.shape[0]
        nb = n // self.batch
        perm_stream = synthetic.Stream(seed, synthetic.TAG_SHUFFLE)
        losses = []
        # The instances are i.i.d. draws, so each epoch visits the fixed
        # batches in a fresh random order (no per-step gathers).
        for ep in range(epochs):
            if schedule == "cosine":
                self.student.set_adam(lr=lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs)))
            order = np.argsort(perm_stream.uniform(nb))
            for b in order:
                sl = slice(int(b) * self.batch, (int(b) + 1) * self.batch)
                loss = self.student.train_step(data.x[sl], data.labels[sl], data.target[sl], data.v_empty)
            losses.append(float(loss.item()))
            if log:
                log(ep, losses[-1])
        self.student.check()
        return losses

    # -- inference --------------------------------------------------------------
    def residuals(self, x32, phi, first: int = 0):
        """Surrogate residual of each instance at its spot-check coalitions
        (pool rows, cycled for calls longer than the pool)."""
        torch = self.torch
        lib = _declare()
        n = x32.shape[0]
        r = torch.empty(n, dtype=torch.float32, device="cuda")
        x64 = x32.double()
        for s in range(0, n, self.batch):
            e = min(n, s + self.batch)
            c = self.coal_pool_dev[:e - s]
            vcoal = torch.empty(c.shape, dtype=torch.float32, device="cuda")
            self._values_listed(x64[s:e], c, vcoal, self.tc)
            _check(lib.tt_fsi_surrogate_residual(_p(phi[s:e]), e - s, self.n_out, _p(self.masks), _p(c), _p(vcoal),
                                                  self.K, _p(r[s:e]), _stream_ptr()), "tt_fsi_surrogate_residual")
        return r

    def calibrate(self, data: Dataset, quantile: float = 0.99):
        """Fallback threshold: the given quantile of the student's residual on
        held-out instances."""
        phi = self.predict_raw(data.x, data.target)
        r = self.residuals(data.x, phi).cpu().numpy()
        self.tau = float(np.quantile(r, quantile))
        return self.tau

    def predict_raw(self, x32, target):
        torch = self.torch
        n = x32.shape[0]
        out = torch.empty((n, self.n_out), dtype=torch.float32, device="cuda")
        for s in range(0, n, self.batch):
            e = min(n, s + self.batch)
            self.student.predict(x32[s:e].contiguous(), target[s:e].contiguous(), self.v_empty, out=out[s:e])
        return out

    def explain(self, x32, target=None, first: int = 0):
        """Student scores with the residual check; failing instances are
        recomputed exactly.  Returns (phi float64 [n, n_out], fallback mask)."""
        torch = self.torch
        if target is None:
            target = self.targets(x32.double())
        phi = self.predict_raw(x32, target)
        r = self.residuals(x32, phi, first=first)
        fb = r > self.tau
        out = phi.double()
        idx = torch.nonzero(fb).flatten()
        if idx.numel():
            out[idx] = self.exact(x32[idx].double())
        return out, fb

