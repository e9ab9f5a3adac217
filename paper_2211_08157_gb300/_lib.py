"""Build and load ``libgod.so`` (the sm_103a CUDA library behind include/god.h).

The shared library is compiled in-tree with nvcc (one ``-gencode`` for
sm_103a, translation units compiled in parallel) into
``paper_2211_08157_gb300/libgod.so``. There is no fallback: when the library
is missing or cannot load, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgod.so")
INCLUDE = os.path.join(ROOT, "include")
SOURCES = ["api.cu", "scan.cu", "sketch.cu", "radix.cu", "index.cu", "rmi.cu", "seed.cu", "serve.cu", "vote.cu",
           "segment.cu", "contain.cu", "seedmatch.cu",
           "sketch_seg.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xcompiler", "-Wall", "-I", INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "god.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every translation unit for sm_103a and link libgod.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, err in results:
            if err.strip():
                print(err)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *[o for o, _ in results], "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


_lock = threading.Lock()
_lib = None


class GodError(RuntimeError):
    def __init__(self, rc: int, msg: str):
        super().__init__(f"{msg} (rc={rc})")
        self.rc = rc


class Params(C.Structure):
    _fields_ = [("index_kind", C.c_int), ("pa_t", C.c_uint32), ("rmi_leaf_bits", C.c_int),
                ("rmi_eps_max", C.c_uint32), ("rmi_root", C.c_int), ("rmi_train_steps", C.c_int),
                ("rmi_train_samples", C.c_uint32), ("tune", C.c_int)]


class SeedOpts(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("pa_t", C.c_uint32), ("via", C.c_int), ("shifts_out", C.c_void_p),
                ("seg_len", C.c_uint32)]


class IndexInfo(C.Structure):
    _fields_ = [("ref_len", C.c_uint64), ("n_minimizers", C.c_uint64), ("n_keys", C.c_uint64),
                ("n_entries", C.c_uint64), ("ht_capacity", C.c_uint64), ("k", C.c_int), ("w", C.c_int),
                ("p", C.c_int), ("x", C.c_int), ("max_occ", C.c_uint32), ("has_learned", C.c_int),
                ("rmi_leaves", C.c_uint32), ("rmi_fallback_leaves", C.c_uint32), ("rmi_mean_eps", C.c_double),
                ("rmi_max_eps", C.c_uint32), ("rmi_fallback_key_frac", C.c_double), ("rmi_final_loss", C.c_float),
                ("device_bytes", C.c_uint64)]


class VoteParams(C.Structure):
    _fields_ = [("D", C.c_uint32), ("V", C.c_uint32), ("max_out", C.c_uint32)]


class ContainParams(C.Structure):
    _fields_ = [("pattern", C.c_char_p), ("k", C.c_int), ("w", C.c_int), ("max_occ", C.c_uint32),
                ("pa_t", C.c_uint32), ("D", C.c_uint32), ("V", C.c_uint32), ("index_kind", C.c_int),
                ("batch_bases", C.c_uint64)]


class ServerConfig(C.Structure):
    _fields_ = [("slots", C.c_int), ("mem_budget", C.c_uint64), ("max_batch_bases", C.c_uint64)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("batches", C.c_uint64),
                ("max_inflight_batches", C.c_uint64), ("merged_requests", C.c_uint64), ("rejected", C.c_uint64),
                ("gather_s", C.c_double), ("pin_alloc_s", C.c_double), ("device_s", C.c_double),
                ("copy_back_s", C.c_double)]


# name -> (restype, argtypes); every symbol declared in include/god.h
P_, U64, U32, I32 = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int
SIGNATURES = {
    "god_strerror": (C.c_char_p, [I32]),
    "god_last_error": (C.c_char_p, []),
    "god_params_init": (None, [C.POINTER(Params)]),
    "god_build_index": (I32, [P_, U64, C.c_char_p, I32, I32, U32, C.POINTER(P_)]),
    "god_build_index_ex": (I32, [P_, U64, C.c_char_p, I32, I32, U32, C.POINTER(Params), P_, C.POINTER(P_)]),
    "god_index_get_info": (I32, [P_, C.POINTER(IndexInfo)]),
    "god_index_export": (I32, [P_, P_, P_, P_]),
    "god_index_lookup": (I32, [P_, P_, U64, I32, P_, P_, P_]),
    "god_seed": (I32, [P_, P_, P_, U32, C.POINTER(P_), C.POINTER(U64)]),
    "god_seed_opts_init": (None, [C.POINTER(SeedOpts)]),
    "god_seed_into": (I32, [P_, P_, P_, U32, P_, U64, C.POINTER(U64), C.POINTER(SeedOpts)]),
    "god_seed_device": (I32, [P_, P_, P_, U32, C.POINTER(P_), C.POINTER(U64), C.POINTER(SeedOpts)]),
    "god_sketch": (I32, [P_, U64, C.c_char_p, U32, I32, I32, P_, P_, P_, U64, C.POINTER(U64), P_]),
    "god_sketch_noalloc": (I32, [P_, U64, C.c_char_p, U32, I32, I32, P_, U64, C.POINTER(U64), P_]),
    "god_rmi_root_grad": (I32, [P_, I32, P_, P_, U64, P_, P_]),
    "god_vote": (I32, [P_, U64, P_, U32, C.POINTER(VoteParams), P_, P_, P_]),
    "god_contain_params_init": (None, [C.POINTER(ContainParams)]),
    "god_contain": (I32, [P_, P_, U32, P_, U32, P_, P_, U32, C.POINTER(ContainParams), P_, P_, P_, P_, P_]),
    "god_seed_match": (I32, [P_, P_, U32, C.c_char_p, C.c_char_p, I32, I32, P_, P_, P_, P_]),
    "god_free": (None, [P_]),
    "god_launch_count": (U64, []),
    "god_prof_enable": (None, [I32]),
    "god_prof_reset": (None, []),
    "god_prof_timeline": (I32, [C.c_char_p, U64]),
    "god_prof_report": (I32, [C.c_char_p, U64]),
    "god_set_graphs": (None, [I32]),
    "god_autotune_report": (I32, [C.c_char_p, U64]),
    "god_server_config_init": (None, [C.POINTER(ServerConfig)]),
    "god_server_create": (I32, [P_, C.POINTER(ServerConfig), C.POINTER(P_)]),
    "god_server_submit": (I32, [P_, P_, P_, U32, C.POINTER(U64)]),
    "god_server_wait": (I32, [P_, U64, I32, C.POINTER(P_), C.POINTER(U64), C.POINTER(C.c_double)]),
    "god_server_get_stats": (I32, [P_, C.POINTER(ServerStats)]),
    "god_server_destroy": (I32, [P_]),
}


def load(build_if_missing: bool = True):
    """Load libgod.so (building it first when absent or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                build()
            if not os.path.exists(LIB):
                raise RuntimeError("libgod.so is not built; call paper_2211_08157_gb300.build()")
            L = C.CDLL(LIB)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(rc: int):
    if rc != 0:
        L = load()
        raise GodError(rc, f"{L.god_strerror(rc).decode()}: {L.god_last_error().decode()}")
