"""GB300-native Faithful Shapley Interactions (TT-FSI hot path).

The compute runs in the CUDA kernels of ``csrc/`` behind the C ABI of
``include/tt_fsi.h``; this module only marshals PyTorch tensors (device
memory and the current CUDA stream) into those calls.  There is no CPU
fallback: without the native library or a CUDA device every call raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import native

ARITH = {"exact": 0, "f64": 1, "f32": 2}
# interaction indices (tt_fsi_index)
INDEX = {"fsi": 0, "sii": 1, "bii": 2, "stii": 3, "ksii": 4}
STATUS = {
    0: "ok", 1: "invalid argument", 2: "unsupported", 3: "out of memory", 4: "CUDA error",
    5: "device wait timed out", 6: "non-finite input", 7: "self-check failed",
}


class FsiError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {STATUS.get(self.status, 'unknown')} (status {self.status})")


def _check(status: int, what: str):
    if status != 0:
        if status in (3, 4):
            what = f"{what} [{native.load().tt_fsi_last_cuda_error().decode()}]"
        raise FsiError(status, what)


def num_scores(d: int, ell: int) -> int:
    n = native.load().tt_fsi_num_scores(d, ell)
    if n < 0:
        raise ValueError("need 1 <= d <= 62 and ell >= 1")
    return int(n)


def score_masks(d: int, ell: int) -> np.ndarray:
    out = np.empty(num_scores(d, ell), dtype=np.uint64)
    _check(native.load().tt_fsi_score_masks(d, ell, out.ctypes.data), "tt_fsi_score_masks")
    return out


def plan_weights(d: int, ell: int, index: str = "fsi"):
    """Host introspection of the exact plan's combined weights (no GPU):
    returns (num [S1, P1, Q1] int64, den [S1] int64, b, h) with
    omega_s(p, q) = num[s, p, q] / den[s] (see tt_fsi_plan_weights)."""
    lib = native.load()
    dims = np.zeros(5, dtype=np.int32)
    _check(lib.tt_fsi_plan_weights(d, ell, INDEX[index], None, None, ctypes.c_void_p(dims.ctypes.data)),
           "tt_fsi_plan_weights")
    S1, P1, Q1, b, h = (int(x) for x in dims)
    num = np.zeros(S1 * P1 * Q1, dtype=np.int64)
    den = np.zeros(S1, dtype=np.int64)
    _check(lib.tt_fsi_plan_weights(d, ell, INDEX[index], ctypes.c_void_p(num.ctypes.data),
                                   ctypes.c_void_p(den.ctypes.data), ctypes.c_void_p(dims.ctypes.data)),
           "tt_fsi_plan_weights")
    return num.reshape(S1, P1, Q1), den, b, h


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """tt_fsi_plan(d, l): tables and scratch for FSI of order ``ell`` on
    ``d``-player games, for batches of up to ``max_batch`` games."""

    def __init__(self, d: int, ell: int, arith: str = "exact", max_batch: int = 1, index: str = "fsi",
                 site_sweep: bool = False, precontract: bool = False):
        """site_sweep: contract every tile site by site (the paper's sweep),
        the comparison variant of the default 4-bit register groups;
        precontract: the same sweep of the precontracted operator on v, with
        the Moebius step folded into each site's core (no Moebius pass)."""
        self._lib = native.load()
        self.d, self.ell, self.arith, self.max_batch, self.index = d, ell, arith, max_batch, index
        h = ctypes.c_void_p()
        _check(self._lib.tt_fsi_plan_create_ex(d, ell, INDEX[index], ARITH[arith], max_batch,
                                               (1 if site_sweep else 0) | (2 if precontract else 0),
                                               ctypes.byref(h)), "tt_fsi_plan_create_ex")
        self._h = h
        self.n_scores = num_scores(d, ell)

    @property
    def handle(self):
        return self._h

    @property
    def tile_bits(self) -> int:
        return int(self._lib.tt_fsi_plan_tile_bits(self._h))

    @property
    def scratch_bytes(self) -> int:
        return int(self._lib.tt_fsi_plan_scratch_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tt_fsi_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, v, out=None, stream=None):
        """phi = FSI(v) for v [B, 2^d] on the GPU (float64, float32 for the
        f32 plan).  Returns [B, n_scores] on the same device."""
        import torch
        dt = torch.float32 if self.arith == "f32" else torch.float64
        if v.dim() == 1:
            v = v.unsqueeze(0)
        if not v.is_cuda or v.dtype != dt or v.shape[-1] != (1 << self.d):
            raise ValueError(f"v must be a CUDA {dt} tensor of shape [B, 2^{self.d}]")
        v = v.contiguous()
        B = v.shape[0]
        if out is None:
            out = torch.empty((B, self.n_scores), dtype=dt, device=v.device)
        _check(self._lib.tt_fsi_apply(self._h, ctypes.c_void_p(v.data_ptr()), B,
                                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
               "tt_fsi_apply")
        return out

    def apply_host(self, v, out=None, stream=None):
        """End to end from host memory: v [B, 2^d] CPU tensor (page-locked
        copies fastest) -> phi [B, n_scores] CPU tensor; the input moves to
        the device in chunks that overlap the compute."""
        import torch
        dt = torch.float32 if self.arith == "f32" else torch.float64
        if v.dim() == 1:
            v = v.unsqueeze(0)
        if v.is_cuda or v.dtype != dt or v.shape[-1] != (1 << self.d):
            raise ValueError(f"v must be a CPU {dt} tensor of shape [B, 2^{self.d}]")
        v = v.contiguous()
        B = v.shape[0]
        if out is None:
            out = torch.empty((B, self.n_scores), dtype=dt, pin_memory=v.is_pinned())
        if out.is_cuda or out.dtype != dt or tuple(out.shape) != (B, self.n_scores) or not out.is_contiguous():
            raise ValueError(f"out must be a contiguous CPU {dt} tensor of shape [B, {self.n_scores}]")
        _check(self._lib.tt_fsi_apply_host(self._h, ctypes.c_void_p(v.data_ptr()), B,
                                           ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
               "tt_fsi_apply_host")
        return out

    def set_host_zero_copy(self, enable: bool = True):
        """apply_host on page-locked input: read it in place (default) or
        always through staged copies."""
        _check(self._lib.tt_fsi_plan_set_host_zero_copy(self._h, 1 if enable else 0),
               "tt_fsi_plan_set_host_zero_copy")

    def set_host_chunk(self, games: int = 0):
        """Games per host-transfer chunk of apply_host (0: automatic)."""
        _check(self._lib.tt_fsi_plan_set_host_chunk(self._h, games), "tt_fsi_plan_set_host_chunk")

    def check(self, stream=None):
        _check(self._lib.tt_fsi_plan_check(self._h, _stream_ptr(stream)), "tt_fsi_plan_check")

    def set_schedule(self, fused: bool = False, tiles_per_item: int = 1, scores_per_item: int = 64):
        """Tile launch + combine launch (default) or one fused persistent
        launch (fast path only; results are identical)."""
        _check(self._lib.tt_fsi_plan_set_schedule(self._h, int(bool(fused)), tiles_per_item,
                                                  scores_per_item), "tt_fsi_plan_set_schedule")

    def set_wait_limit(self, polls: int, inject_missing: bool = False):
        """Bound on the fused schedule's device wait; inject_missing makes
        every wait run out (test hook of the timeout path)."""
        _check(self._lib.tt_fsi_plan_set_wait_limit(self._h, polls, int(bool(inject_missing))),
               "tt_fsi_plan_set_wait_limit")


def fsi(v, d: int, ell: int, arith: str = "exact", index: str = "fsi"):
    """One-shot interaction scores (FSI by default; index "sii", "bii",
    "stii" or "ksii" for the other indices) of v [B, 2^d] (CUDA tensor)."""
    B = 1 if v.dim() == 1 else v.shape[0]
    p = Plan(d, ell, arith, max_batch=max(1, B), index=index)
    try:
        out = p.apply(v)
        p.check()
        return out
    finally:
        p.close()


class _Mlp(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("h1", ctypes.c_int), ("h2", ctypes.c_int),
                ("W1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("W2", ctypes.c_void_p),
                ("b2", ctypes.c_void_p), ("W3", ctypes.c_void_p), ("b3", ctypes.c_double),
                ("W1f", ctypes.c_void_p), ("b1f", ctypes.c_void_p), ("W2f", ctypes.c_void_p),
                ("b2f", ctypes.c_void_p), ("W3f", ctypes.c_void_p)]


class DeviceMLP:
    """Float64 copies of an MLP's weights on a CUDA device, in the layout of
    tt_fsi_mlp (W1 [h1, d], W2 [h2, h1], W3 [h2], row-major)."""

    def __init__(self, mlp, device="cuda"):
        import torch
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)
        self.W1, self.b1 = f(mlp.W1), f(mlp.b1)
        self.W2, self.b2 = f(mlp.W2), f(mlp.b2)
        self.W3 = f(np.asarray(mlp.W3).reshape(-1))
        self.b3 = float(np.asarray(mlp.b3).reshape(-1)[0])
        self.h1, self.d = self.W1.shape
        self.h2 = self.W2.shape[0]
        self._f = [t.float().contiguous() for t in (self.W1, self.b1, self.W2, self.b2, self.W3)]
        self._s = _Mlp(self.d, self.h1, self.h2, self.W1.data_ptr(), self.b1.data_ptr(),
                       self.W2.data_ptr(), self.b2.data_ptr(), self.W3.data_ptr(), self.b3,
                       *[t.data_ptr() for t in self._f])

    @property
    def struct(self):
        return self._s


def masked_game_into(mlp, x, baseline, out, stream=None):
    """v[b, S] = f(x[b] on S, baseline elsewhere) for all 2^d coalitions,
    written into ``out`` ([B, 2^d], float64 or float32) by the CUDA kernel."""
    import torch
    dm = mlp if isinstance(mlp, DeviceMLP) else DeviceMLP(mlp, out.device)
    x = x.to(device=out.device, dtype=torch.float64).contiguous()
    baseline = baseline.to(device=out.device, dtype=torch.float64).contiguous()
    if x.dim() == 1:
        x = x.unsqueeze(0)
    B = x.shape[0]
    if out.shape != (B, 1 << dm.d) or not out.is_contiguous():
        raise ValueError("out must be a contiguous [B, 2^d] tensor")
    f32 = 1 if out.dtype == torch.float32 else 0
    if not f32 and out.dtype != torch.float64:
        raise ValueError("out must be float64 or float32")
    _check(native.load().tt_fsi_masked_game(ctypes.byref(dm.struct), ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(baseline.data_ptr()), B,
                                            ctypes.c_void_p(out.data_ptr()), f32, _stream_ptr(stream)),
           "tt_fsi_masked_game")
    return out


def masked_game_tc(mlp, x, baseline, coalitions=None, out=None, stream=None):
    """Value function on the tensor cores (BF16 layer-2 products, FP32
    out): every coalition ([B, 2^d]) or, given ``coalitions`` [B, K] uint32
    masks, those only ([B, K]).  Needs hidden widths 128.  ``baseline`` [d]
    is one reference input; [n, d] are n background rows (the interventional
    value function: the mean of f over them)."""
    import torch
    dm = mlp if isinstance(mlp, DeviceMLP) else DeviceMLP(mlp)
    dev = dm.W1.device
    x = torch.as_tensor(x).to(device=dev, dtype=torch.float64).contiguous()
    if x.dim() == 1:
        x = x.unsqueeze(0)
    baseline = torch.as_tensor(baseline).to(device=dev, dtype=torch.float64).contiguous()
    B = x.shape[0]
    if coalitions is None:
        shape, cptr, K = (B, 1 << dm.d), None, 0
    else:
        c = torch.as_tensor(coalitions)
        if c.dtype != torch.int32:
            c = torch.as_tensor(np.ascontiguousarray(np.asarray(coalitions, dtype=np.uint32)).view(np.int32))
        c = c.to(dev).contiguous()
        if c.dim() != 2 or c.shape[0] != B:
            raise ValueError("coalitions must be [B, K]")
        shape, cptr, K = tuple(c.shape), ctypes.c_void_p(c.data_ptr()), int(c.shape[1])
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=dev)
    if tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous float32 tensor of shape {shape}")
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    n_bg = 1 if baseline.dim() == 1 else baseline.shape[0]
    if baseline.shape[-1] != dm.d:
        raise ValueError("baseline rows must have d entries")
    _check(native.load().tt_fsi_masked_game_tc_interventional(
        ctypes.byref(dm.struct), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(baseline.data_ptr()), n_bg, B,
        cptr, K, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(err.data_ptr()), _stream_ptr(stream)),
        "tt_fsi_masked_game_tc_interventional")
    if int(err.item()) != 0:
        raise FsiError(5, "tt_fsi_masked_game_tc")
    return out


def masked_game_interventional(mlp, x, background, dtype=None, stream=None):
    """Interventional value function (the mean of f over the rows of
    ``background`` [n, d] for the absent features) for all 2^d coalitions,
    [B, 2^d] float64 (or float32) by the CUDA kernel."""
    import torch
    dm = mlp if isinstance(mlp, DeviceMLP) else DeviceMLP(mlp)
    dev = dm.W1.device
    x = torch.as_tensor(x).to(device=dev, dtype=torch.float64).contiguous()
    if x.dim() == 1:
        x = x.unsqueeze(0)
    bg = torch.as_tensor(background).to(device=dev, dtype=torch.float64).contiguous()
    if bg.dim() != 2 or bg.shape[1] != dm.d:
        raise ValueError("background must be [n, d]")
    B = x.shape[0]
    dt = dtype or torch.float64
    out = torch.empty((B, 1 << dm.d), dtype=dt, device=dev)
    _check(native.load().tt_fsi_masked_game_interventional(
        ctypes.byref(dm.struct), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(bg.data_ptr()), bg.shape[0], B,
        ctypes.c_void_p(out.data_ptr()), 1 if dt == torch.float32 else 0, _stream_ptr(stream)),
        "tt_fsi_masked_game_interventional")
    return out


def masked_game(mlp, x, baseline, dtype=None, stream=None):
    import torch
    dm = mlp if isinstance(mlp, DeviceMLP) else DeviceMLP(mlp)
    x = torch.as_tensor(x)
    B = 1 if x.dim() == 1 else x.shape[0]
    out = torch.empty((B, 1 << dm.d), dtype=dtype or torch.float64, device=dm.W1.device)
    return masked_game_into(dm, torch.as_tensor(x, device=dm.W1.device),
                            torch.as_tensor(baseline, device=dm.W1.device), out, stream)


class _Game(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("ell", ctypes.c_int), ("v_offset", ctypes.c_int64),
                ("phi_offset", ctypes.c_int64)]


class Batch:
    """Many games of uneven size (d, l) in one persistent launch.  ``games``
    is a sequence of (d, ell, v_offset, phi_offset), offsets in elements of
    the batch's packed value and score buffers."""

    def __init__(self, games, arith: str = "exact", index: str = "fsi"):
        self._lib = native.load()
        self.arith, self.index = arith, index
        arr = (_Game * len(games))(*[_Game(int(d), int(l), int(vo), int(po)) for d, l, vo, po in games])
        h = ctypes.c_void_p()
        _check(self._lib.tt_fsi_batch_create_index(ctypes.cast(arr, ctypes.c_void_p), len(games),
                                                   ARITH[arith], INDEX[index], ctypes.byref(h)),
               "tt_fsi_batch_create_index")
        self._h = h
        self.n_games = len(games)

    @classmethod
    def from_ragged(cls, g, arith: str = "exact", index: str = "fsi"):
        return cls([(int(g.d[k]), int(g.ell[k]), int(g.v_off[k]), int(g.phi_off[k]))
                    for k in range(len(g.d))], arith, index)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tt_fsi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, v, phi, stream=None):
        _check(getattr(self._lib, name)(self._h, ctypes.c_void_p(v.data_ptr()),
                                        ctypes.c_void_p(phi.data_ptr()), _stream_ptr(stream)), name)
        return phi

    def apply(self, v, phi, stream=None):
        """One persistent launch over every game (the batched path)."""
        return self._call("tt_fsi_batch_apply", v, phi, stream)

    def apply_per_game(self, v, phi, stream=None):
        return self._call("tt_fsi_batch_apply_per_game", v, phi, stream)

    def apply_graph(self, v, phi, stream=None):
        return self._call("tt_fsi_batch_apply_graph", v, phi, stream)

    def autotune(self, v, phi, stream=None):
        t, c = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.tt_fsi_batch_autotune(self._h, ctypes.c_void_p(v.data_ptr()),
                                               ctypes.c_void_p(phi.data_ptr()), _stream_ptr(stream),
                                               ctypes.byref(t), ctypes.byref(c)), "tt_fsi_batch_autotune")
        return t.value, c.value

    def set_schedule(self, tiles_per_item: int, scores_per_item: int):
        _check(self._lib.tt_fsi_batch_set_schedule(self._h, tiles_per_item, scores_per_item),
               "tt_fsi_batch_set_schedule")

    def set_wait_limit(self, polls: int, inject_missing_tile: bool = False):
        _check(self._lib.tt_fsi_batch_set_wait_limit(self._h, polls, 1 if inject_missing_tile else 0),
               "tt_fsi_batch_set_wait_limit")

    def check(self, stream=None):
        _check(self._lib.tt_fsi_batch_check(self._h, _stream_ptr(stream)), "tt_fsi_batch_check")
