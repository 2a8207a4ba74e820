"""Build and load the native library (CUDA kernels for sm_103a + C ABI).

The library is compiled in-tree with nvcc into ``_build/libttfsi.so`` and
loaded with ctypes.  Nothing here falls back to another implementation: if
the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libttfsi.so")
INCLUDE = os.path.join(_ROOT, "include")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

_lock = threading.Lock()
_lib = None


def sources():
    out = []
    for name in sorted(os.listdir(_CSRC)):
        if name.endswith((".cu", ".cpp")):
            out.append(os.path.join(_CSRC, name))
    return out


def _deps():
    files = sources()
    for name in os.listdir(_CSRC):
        if name.endswith((".h", ".cuh")):
            files.append(os.path.join(_CSRC, name))
    for name in os.listdir(INCLUDE):
        files.append(os.path.join(INCLUDE, name))
    return files


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(f) > t for f in _deps())


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in csrc/ for sm_103a (in parallel) and
    link them into one shared library."""
    with _lock:
        if not force and not _stale():
            return LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        common = ["-std=c++17", "-O3", "-lineinfo", ARCH, "-Xcompiler", "-fPIC",
                  "-I" + INCLUDE, "-I" + _CSRC]

        def compile_one(src):
            obj = os.path.join(_BUILD, os.path.basename(src) + ".o")
            cmd = [nvcc()] + common + ["-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                print(r.stdout, r.stderr)
            return obj

        srcs = sources()
        with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
            objs = list(ex.map(compile_one, srcs))
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        cmd = [nvcc(), ARCH, "-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB_PATH)
        return LIB_PATH


def load():
    """Load (building first if needed) the native library; raises if that
    is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    lib = ctypes.CDLL(path)
    _declare(lib)
    _lib = lib
    return lib


def _declare(lib):
    c = ctypes
    i, i64, u64p, vp, sz = c.c_int, c.c_int64, c.POINTER(c.c_uint64), c.c_void_p, c.c_size_t
    lib.tt_fsi_num_scores.restype = i64
    lib.tt_fsi_num_scores.argtypes = [i, i]
    lib.tt_fsi_score_masks.restype = i
    lib.tt_fsi_score_masks.argtypes = [i, i, vp]
    lib.tt_fsi_plan_create.restype = i
    lib.tt_fsi_plan_create.argtypes = [i, i, i, i64, c.POINTER(vp)]
    lib.tt_fsi_plan_create_index.restype = i
    lib.tt_fsi_plan_create_index.argtypes = [i, i, i, i, i64, c.POINTER(vp)]
    lib.tt_fsi_plan_create_ex.restype = i
    lib.tt_fsi_plan_create_ex.argtypes = [i, i, i, i, i64, c.c_uint, c.POINTER(vp)]
    lib.tt_fsi_batch_create_index.restype = i
    lib.tt_fsi_batch_create_index.argtypes = [vp, i64, i, i, c.POINTER(vp)]
    lib.tt_fsi_plan_destroy.restype = None
    lib.tt_fsi_plan_destroy.argtypes = [vp]
    lib.tt_fsi_plan_scratch_bytes.restype = sz
    lib.tt_fsi_plan_scratch_bytes.argtypes = [vp]
    lib.tt_fsi_plan_tile_bits.restype = i
    lib.tt_fsi_plan_tile_bits.argtypes = [vp]
    lib.tt_fsi_apply.restype = i
    lib.tt_fsi_apply.argtypes = [vp, vp, i64, vp, vp]
    lib.tt_fsi_plan_check.restype = i
    lib.tt_fsi_plan_check.argtypes = [vp, vp]
    lib.tt_fsi_plan_set_schedule.restype = i
    lib.tt_fsi_plan_set_schedule.argtypes = [vp, i, i, i]
    lib.tt_fsi_plan_set_wait_limit.restype = i
    lib.tt_fsi_plan_set_wait_limit.argtypes = [vp, c.c_longlong, i]
    lib.tt_fsi_last_cuda_error.restype = c.c_char_p
    lib.tt_fsi_last_cuda_error.argtypes = []
    lib.tt_fsi_status_string.restype = c.c_char_p
    lib.tt_fsi_status_string.argtypes = [i]
    lib.tt_fsi_apply_host.restype = i
    lib.tt_fsi_apply_host.argtypes = [vp, vp, i64, vp, vp]
    lib.tt_fsi_plan_set_host_chunk.restype = i
    lib.tt_fsi_plan_set_host_chunk.argtypes = [vp, i64]
    lib.tt_fsi_plan_set_host_zero_copy.restype = i
    lib.tt_fsi_plan_set_host_zero_copy.argtypes = [vp, i]
    lib.tt_fsi_plan_weights.restype = i
    lib.tt_fsi_plan_weights.argtypes = [i, i, i, vp, vp, vp]
    lib.tt_fsi_plan_profile.restype = i
    lib.tt_fsi_plan_profile.argtypes = [vp, i]
    lib.tt_fsi_plan_profile_read.restype = i
    lib.tt_fsi_plan_profile_read.argtypes = [vp, c.POINTER(c.c_double), c.POINTER(c.c_double),
                                             c.POINTER(i64)]
    lib.tt_fsi_masked_game.restype = i
    lib.tt_fsi_masked_game.argtypes = [vp, vp, vp, i64, vp, i, vp]
    lib.tt_fsi_masked_game_tc.restype = i
    lib.tt_fsi_masked_game_tc.argtypes = [vp, vp, vp, i64, vp, i, vp, vp, vp]
    lib.tt_fsi_masked_game_tc_interventional.restype = i
    lib.tt_fsi_masked_game_tc_interventional.argtypes = [vp, vp, vp, i, i64, vp, i, vp, vp, vp]
    lib.tt_fsi_masked_game_interventional.restype = i
    lib.tt_fsi_masked_game_interventional.argtypes = [vp, vp, vp, i, i64, vp, i, vp]
    lib.tt_fsi_apply_noalloc.restype = i
    lib.tt_fsi_apply_noalloc.argtypes = [i, i, vp, i64, vp, vp]
    for name in ("tt_fsi_batch_apply", "tt_fsi_batch_apply_per_game", "tt_fsi_batch_apply_graph"):
        getattr(lib, name).restype = i
        getattr(lib, name).argtypes = [vp, vp, vp, vp]
    lib.tt_fsi_batch_create.restype = i
    lib.tt_fsi_batch_create.argtypes = [vp, i64, i, c.POINTER(vp)]
    lib.tt_fsi_batch_destroy.restype = None
    lib.tt_fsi_batch_destroy.argtypes = [vp]
    lib.tt_fsi_batch_autotune.restype = i
    lib.tt_fsi_batch_autotune.argtypes = [vp, vp, vp, vp, c.POINTER(i), c.POINTER(i)]
    lib.tt_fsi_batch_set_schedule.restype = i
    lib.tt_fsi_batch_set_schedule.argtypes = [vp, i, i]
    lib.tt_fsi_batch_set_wait_limit.restype = i
    lib.tt_fsi_batch_set_wait_limit.argtypes = [vp, c.c_longlong, i]
    lib.tt_fsi_batch_check.restype = i
    lib.tt_fsi_batch_check.argtypes = [vp, vp]
    lib.tt_fsi_peak_launch.restype = i
    lib.tt_fsi_peak_launch.argtypes = [i, i, i, vp, c.POINTER(i64), vp]
    lib.tt_fsi_gemm_bf16.restype = i
    lib.tt_fsi_gemm_bf16.argtypes = [vp, i, vp, i, i, i, i, vp, i, vp, i, vp, i, vp, i, vp, i, vp, vp]
    for name, args, res in EXTRA_SIGNATURES:
        fn = getattr(lib, name, None)
        if fn is not None:
            fn.argtypes = args
            fn.restype = res


# Further entry points register their signatures here as they are added.
EXTRA_SIGNATURES = []


def exported_symbols():
    """Names declared extern "C" in include/*.h (parsed from the headers)."""
    import re
    names = []
    for name in sorted(os.listdir(INCLUDE)):
        if not name.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, name)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(tt_fsi_[a-z0-9_]+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))
