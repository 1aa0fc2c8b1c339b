"""GB300 column-density tracer (RAYTHEIA hot path, arXiv 2605.09882).

Thin ctypes binding over the C ABI in include/rt_api.h.  PyTorch supplies
device memory and streams only: every step of the trace runs in the library's
CUDA kernels.  There is no CPU fallback: importing this package without the
built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

__all__ = ["Octree", "Batch", "Paths", "trace_epilogue", "build_amr", "healpix_dirs", "trace_columns", "trace_paths", "trace_columns_adjoint",
           "trace_columns_chunked", "trace_columns_host", "trace_batched", "autotune",
           "Columns", "RTError", "MODE_FP64", "MODE_F32_KAHAN", "set_launch", "lib_path"]

MODE_FP64, MODE_F32_KAHAN = 0, 1
F32, F64 = 0, 1
STATUS = {0: "RT_OK", 1: "RT_ERR_ARG", 2: "RT_ERR_UNSORTED", 3: "RT_ERR_MISALIGNED",
          4: "RT_ERR_OVERLAP_OR_GAP", 5: "RT_ERR_SOURCE_OUTSIDE", 6: "RT_ERR_STEP_LIMIT",
          7: "RT_ERR_NONFINITE", 8: "RT_ERR_CUDA", 9: "RT_ERR_OOM", 10: "RT_ERR_LOOKUP_MISS"}


class RTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class CloudDesc(C.Structure):
    _fields_ = [("tree", C.c_void_p), ("d_src", C.c_void_p), ("n_src", C.c_int64), ("nside", C.c_int),
                ("n_species", C.c_int), ("d_dens", C.c_void_p), ("dens_dtype", C.c_int),
                ("reserved", C.c_int), ("d_out", C.c_void_p)]


class Epilogue(C.Structure):
    _fields_ = [("kind", C.c_int), ("reserved", C.c_int), ("weights", C.c_double * 8), ("a", C.c_double),
                ("gamma", C.c_double), ("d_coef", C.c_void_p)]


EPI_AV_EFF, EPI_BETA, EPI_ATTENUATION = 1, 2, 3


class Stats(C.Structure):
    _fields_ = [("rays", C.c_uint64), ("segments", C.c_uint64), ("exit_fallbacks", C.c_uint64),
                ("lookup_fallbacks", C.c_uint64), ("status", C.c_int32), ("gathered", C.c_int32),
                ("fault_ray", C.c_int64)]


def lib_path() -> str:
    return _build.LIB


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"the CUDA library {path} is not built; run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    P, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    lib.rt_build_octree.argtypes = [P, P, i64, P, P, C.POINTER(P)]
    lib.rt_destroy_octree.argtypes = [P]
    lib.rt_destroy_octree.restype = None
    lib.rt_healpix_dirs.argtypes = [i32, P]
    lib.rt_trace_columns.argtypes = [P, P, i64, i32, P, i32, i32, i32, P, P]
    lib.rt_trace_paths.argtypes = [P, P, i64, i32, i32, P, P, P]
    lib.rt_trace_columns_adjoint.argtypes = [P, P, i64, i32, P, i32, i32, P, i32, P]
    lib.rt_get_stats.argtypes = [P, C.POINTER(Stats), P]
    lib.rt_reset_stats.argtypes = [P, P]
    lib.rt_set_step_cap.argtypes = [P, i64]
    lib.rt_set_launch.argtypes = [i32, i32, i32]
    lib.rt_set_lookup.argtypes = [P, i32]
    lib.rt_set_table_cap.argtypes = [i32]
    lib.rt_octree_info.argtypes = [P, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32)]
    lib.rt_last_error.restype = C.c_char_p
    lib.rt_batch_create.argtypes = [P, i32, i32, C.POINTER(P)]
    lib.rt_batch_launch.argtypes = [P, P]
    lib.rt_batch_stats.argtypes = [P, C.POINTER(Stats), P]
    lib.rt_batch_reset_stats.argtypes = [P, P]
    lib.rt_batch_destroy.argtypes = [P]
    lib.rt_batch_destroy.restype = None
    lib.rt_batch_autotune.argtypes = [P, C.c_char_p, C.POINTER(C.c_int * 3), C.POINTER(C.c_double), P]
    lib.rt_trace_batched.argtypes = [P, i32, i32, P]
    lib.rt_autotune.argtypes = [P, i32, i32, C.c_char_p]
    lib.rt_trace_epilogue.argtypes = [P, P, i64, i32, P, i32, i32, i32, C.POINTER(Epilogue), P, P]
    lib.rt_build_amr.argtypes = [P, i32, P, i32, i32, i32, C.c_double, C.c_double, i32, P, P, P, i64,
                                 C.POINTER(i64), P]
    lib.rt_record_paths.argtypes = [P, P, i64, i32, i32, P, C.POINTER(P)]
    lib.rt_paths_info.argtypes = [P, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    lib.rt_paths_columns.argtypes = [P, P, i32, i32, P, P]
    lib.rt_paths_adjoint.argtypes = [P, P, i32, P, P]
    lib.rt_paths_adjoint_ordered.argtypes = [P, P, i32, P, P]
    lib.rt_destroy_paths.argtypes = [P]
    lib.rt_destroy_paths.restype = None
    lib.rt_trace_columns_host.argtypes = [P, P, i64, P, P, i64, i32, P, i32, i32, i32, P, i64,
                                          C.POINTER(Stats), P]
    lib.rt_trace_columns_chunked.argtypes = [P, P, i64, i32, P, i32, i32, i32, P, i32, P, P, P, P]
    lib.rt_trace_columns_host_release.argtypes = []
    lib.rt_trace_columns_host_release.restype = None
    return lib


_lib = _load()


def _check(code: int):
    if code != 0:
        raise RTError(code, _lib.rt_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def healpix_dirs(nside: int) -> np.ndarray:
    """HEALPix pixel centres (RING order) as float64 [12 nside^2][3] (host)."""
    out = np.zeros((12 * nside * nside, 3), dtype=np.float64)
    _check(_lib.rt_healpix_dirs(int(nside), out.ctypes.data_as(C.c_void_p)))
    return out


def set_table_cap(max_level: int = -1):
    """Deepest coarse-table level later Octree builds may use (-1: no cap)."""
    _check(_lib.rt_set_table_cap(int(max_level)))


def set_launch(threads_per_block: int = 0, blocks_per_sm: int = 0, groups_per_pop: int = 0):
    """Launch shape of the persistent kernels (0 = default for each)."""
    _check(_lib.rt_set_launch(int(threads_per_block), int(blocks_per_sm), int(groups_per_pop)))


class Octree:
    """Handle over device-resident sorted Morton keys (int64/uint64) and
    levels (uint8); the tensors are borrowed and kept alive by the handle."""

    def __init__(self, keys, levels, extent=None, stream=None):
        import torch
        if keys.device.type != "cuda" or levels.device.type != "cuda":
            raise ValueError("keys and levels must be CUDA tensors")
        if keys.dtype not in (torch.int64, torch.uint64) or levels.dtype != torch.uint8:
            raise ValueError("keys must be int64/uint64 and levels uint8")
        self.keys = keys.contiguous()
        self.levels = levels.contiguous()
        self.n_leaves = int(self.keys.numel())
        ext = None
        if extent is not None:
            ext = (C.c_int32 * 3)(*[int(e) for e in extent])
        h = C.c_void_p()
        _check(_lib.rt_build_octree(_dptr(self.keys), _dptr(self.levels), self.n_leaves, ext,
                                    _stream(stream), C.byref(h)))
        self._h = h
        n, lm, ul = C.c_int64(), C.c_int32(), C.c_int32()
        _check(_lib.rt_octree_info(self._h, C.byref(n), C.byref(lm), C.byref(ul)))
        self.max_level, self.uniform_level = lm.value, ul.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.rt_destroy_octree(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self, stream=None) -> dict:
        s = Stats()
        _check(_lib.rt_get_stats(self._h, C.byref(s), _stream(stream)))
        return {f: getattr(s, f) for f, _ in Stats._fields_ if f != "reserved"}

    def reset_stats(self, stream=None):
        _check(_lib.rt_reset_stats(self._h, _stream(stream)))

    def set_step_cap(self, cap: int):
        _check(_lib.rt_set_step_cap(self._h, int(cap)))

    def set_lookup(self, use_uniform_index: bool):
        _check(_lib.rt_set_lookup(self._h, 1 if use_uniform_index else 0))


def _mode(mode) -> int:
    if mode in (MODE_FP64, "fp64"):
        return MODE_FP64
    if mode in (MODE_F32_KAHAN, "f32k", "f32_kahan"):
        return MODE_F32_KAHAN
    raise ValueError(f"unknown mode {mode!r}")


def _check_src(src):
    import torch
    if src.device.type != "cuda" or src.dtype != torch.float64 or src.dim() != 2 or src.shape[1] != 3:
        raise ValueError("sources must be a CUDA float64 tensor of shape [n_src, 3]")
    return src.contiguous()


def trace_columns(tree: Octree, src, nside: int, dens, mode="f32k", out=None, stream=None):
    """Columns [n_src][12 nside^2][S]: float32 (F32-Kahan) or float64 (FP64)."""
    import torch
    m = _mode(mode)
    src = _check_src(src)
    dens = dens.contiguous()
    if dens.dim() == 1:
        dens = dens[:, None]
    if dens.dtype not in (torch.float32, torch.float64) or dens.shape[0] != tree.n_leaves:
        raise ValueError("dens must be float32/float64 [n_leaves, S]")
    S = int(dens.shape[1])
    nd = 12 * nside * nside
    odt = torch.float32 if m == MODE_F32_KAHAN else torch.float64
    if out is None:
        out = torch.empty((src.shape[0], nd, S), dtype=odt, device=src.device)
    elif out.dtype != odt or tuple(out.shape) != (src.shape[0], nd, S) or not out.is_contiguous():
        raise ValueError("out has the wrong dtype, shape or layout")
    _check(_lib.rt_trace_columns(tree.handle, _dptr(src), int(src.shape[0]), int(nside), _dptr(dens), S,
                                 F64 if dens.dtype == torch.float64 else F32, m, _dptr(out),
                                 _stream(stream)))
    return out


def trace_columns_chunked(tree: Octree, src, nside: int, dens, n_chunks: int, mode="f32k", mask=None,
                          out=None, paths=False, stream=None):
    """Columns over a chunked contribution grid: the leaves in n_chunks
    Morton-range chunks traced one at a time (densities streamed from a CPU
    tensor, page-locked for overlapped copies, or read in place from a CUDA
    tensor), with every ray's walk carried between chunks; mask (CUDA uint8
    or bool [n_src]) selects the sources inside the cloud, the others get zero
    columns.  Returns the columns, or (columns, nseg, hash) with paths=True."""
    import torch
    m = _mode(mode)
    src = _check_src(src)
    dens = dens.contiguous()
    if dens.dim() == 1:
        dens = dens[:, None]
    if dens.dtype not in (torch.float32, torch.float64) or dens.shape[0] != tree.n_leaves:
        raise ValueError("dens must be float32/float64 [n_leaves, S]")
    S = int(dens.shape[1])
    nd = 12 * nside * nside
    odt = torch.float32 if m == MODE_F32_KAHAN else torch.float64
    if out is None:
        out = torch.empty((src.shape[0], nd, S), dtype=odt, device=src.device)
    if mask is not None:
        mask = mask.to(device=src.device, dtype=torch.uint8).contiguous()
        if mask.numel() != src.shape[0]:
            raise ValueError("mask must have one entry per source")
    nseg = hsh = None
    if paths:
        nseg = torch.empty((src.shape[0], nd), dtype=torch.int32, device=src.device)
        hsh = torch.empty((src.shape[0], nd), dtype=torch.int64, device=src.device)
    _check(_lib.rt_trace_columns_chunked(tree.handle, _dptr(src), int(src.shape[0]), int(nside), _dptr(dens), S,
                                         F64 if dens.dtype == torch.float64 else F32, m, _dptr(mask),
                                         int(n_chunks), _dptr(out), _dptr(nseg), _dptr(hsh), _stream(stream)))
    return (out, nseg, hsh) if paths else out


def trace_columns_host(keys, levels, src, nside: int, dens, mode="f32k", out=None, extent=None,
                       chunk: int = 0, stream=None):
    """Forward trace end to end from host (CPU) tensors: the octree, densities
    and sources are copied in and the columns copied back inside the call,
    in chunks that overlap the copies with the traces (page-locked tensors
    copy fastest).  The device buffers persist between calls until
    trace_columns_host_release().  Returns (columns, statistics dict)."""
    import torch

    def host(t, what, dtypes):
        if isinstance(t, np.ndarray):
            t = torch.from_numpy(t)
        if t.device.type != "cpu" or not t.is_contiguous() or t.dtype not in dtypes:
            raise ValueError(f"{what} must be a contiguous CPU tensor of {dtypes}")
        return t

    m = _mode(mode)
    keys = host(keys, "keys", (torch.int64, torch.uint64))
    levels = host(levels, "levels", (torch.uint8,))
    src = host(src, "src", (torch.float64,))
    dens = host(dens, "dens", (torch.float32, torch.float64))
    if dens.dim() == 1:
        dens = dens[:, None]
    if src.dim() != 2 or src.shape[1] != 3:
        raise ValueError("src must be float64 [n_src, 3]")
    if dens.shape[0] != keys.numel() or levels.numel() != keys.numel():
        raise ValueError("keys, levels and dens must have one row per leaf")
    S = int(dens.shape[1])
    nd = 12 * nside * nside
    odt = torch.float32 if m == MODE_F32_KAHAN else torch.float64
    if out is None:
        out = torch.empty((src.shape[0], nd, S), dtype=odt)
    elif (out.device.type != "cpu" or out.dtype != odt or tuple(out.shape) != (src.shape[0], nd, S)
          or not out.is_contiguous()):
        raise ValueError("out has the wrong device, dtype, shape or layout")
    ext = None
    if extent is not None:
        ext = (C.c_int32 * 3)(*[int(e) for e in extent])
    st = Stats()
    _check(_lib.rt_trace_columns_host(_dptr(keys), _dptr(levels), int(keys.numel()), ext, _dptr(src),
                                      int(src.shape[0]), int(nside), _dptr(dens), S,
                                      F64 if dens.dtype == torch.float64 else F32, m, _dptr(out), int(chunk),
                                      C.byref(st), _stream(stream)))
    return out, {f: getattr(st, f) for f, _ in Stats._fields_}


def trace_columns_host_release():
    """Frees the device buffers trace_columns_host keeps between calls."""
    _lib.rt_trace_columns_host_release()


def trace_paths(tree: Octree, src, nside: int, mode="f32k", stream=None):
    """Per-ray segment counts (int32) and path hashes (int64 bits of uint64)."""
    import torch
    m = _mode(mode)
    src = _check_src(src)
    nd = 12 * nside * nside
    nseg = torch.empty((src.shape[0], nd), dtype=torch.int32, device=src.device)
    hsh = torch.empty((src.shape[0], nd), dtype=torch.int64, device=src.device)
    _check(_lib.rt_trace_paths(tree.handle, _dptr(src), int(src.shape[0]), int(nside), m,
                               _dptr(nseg), _dptr(hsh), _stream(stream)))
    return nseg, hsh


def trace_epilogue(tree: Octree, src, nside: int, dens, kind, weights, a, gamma=3.02, coef=None, mode="f32k",
                   out=None, stream=None):
    """Per-source A_V,eff / escape probability (float64 [n_src]) or per-ray
    attenuation (float64 [n_src][12 nside^2]) computed inside the trace; the
    columns are never written.  kind: "av_eff", "beta" or "attenuation"."""
    import torch
    k = {"av_eff": EPI_AV_EFF, "beta": EPI_BETA, "attenuation": EPI_ATTENUATION}.get(kind, kind)
    m = _mode(mode)
    src = _check_src(src)
    dens = dens.contiguous()
    if dens.dim() == 1:
        dens = dens[:, None]
    S = int(dens.shape[1])
    w = list(weights) + [0.0] * (8 - len(weights))
    e = Epilogue(k, 0, (C.c_double * 8)(*w), float(a), float(gamma), _dptr(coef) if coef is not None else None)
    shape = (src.shape[0], 12 * nside * nside) if k == EPI_ATTENUATION else (src.shape[0],)
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=src.device)
    _check(_lib.rt_trace_epilogue(tree.handle, _dptr(src), int(src.shape[0]), int(nside), _dptr(dens), S,
                                  F64 if dens.dtype == torch.float64 else F32, m, C.byref(e), _dptr(out),
                                  _stream(stream)))
    return out


def build_amr(nref, vals=None, n_pdr=1.0, rel_var=0.01, max_level=None, stream=None):
    """Contribution grid from a uniform source grid in Morton order (8^L
    cells): the split criterion n_max >= n_pdr and (n_max - n_min) / n_max >=
    rel_var, recursively to max_level.  Returns keys (int64), levels (uint8)
    and leaf means ([n_leaves][S], the dtype of vals)."""
    import torch
    n = int(nref.numel())
    L = n.bit_length() - 1
    if n != 1 << L or L % 3:
        raise ValueError("nref must hold 8^level cells")
    L //= 3
    nref = nref.contiguous()
    if vals is not None:
        vals = vals.contiguous()
        if vals.dim() == 1:
            vals = vals[:, None]
    S = 1 if vals is None else int(vals.shape[1])
    vdt = (vals if vals is not None else nref).dtype
    keys = torch.empty(n, dtype=torch.int64, device=nref.device)
    lev = torch.empty(n, dtype=torch.uint8, device=nref.device)
    out = torch.empty((n, S), dtype=vdt, device=nref.device)
    nl = C.c_int64()
    _check(_lib.rt_build_amr(_dptr(nref), F64 if nref.dtype == torch.float64 else F32, _dptr(vals), S,
                             F64 if vdt == torch.float64 else F32, L, float(n_pdr), float(rel_var),
                             L if max_level is None else int(max_level), _dptr(keys), _dptr(lev), _dptr(out), n,
                             C.byref(nl), _stream(stream)))
    m = nl.value
    return keys[:m], lev[:m], out[:m]


class Paths:
    """Recorded (leaf, ds) sequences of every ray of (tree, src, nside, mode);
    columns and adjoints are then evaluated without walking."""

    def __init__(self, tree: Octree, src, nside: int, mode="f32k", stream=None):
        self.mode = _mode(mode)
        self.src = _check_src(src)
        self.nside, self.tree = nside, tree
        h = C.c_void_p()
        _check(_lib.rt_record_paths(tree.handle, _dptr(self.src), int(self.src.shape[0]), int(nside), self.mode,
                                    _stream(stream), C.byref(h)))
        self._h = h

    def info(self) -> dict:
        r, s, b = C.c_int64(), C.c_int64(), C.c_int64()
        _check(_lib.rt_paths_info(self._h, C.byref(r), C.byref(s), C.byref(b)))
        return {"rays": r.value, "segments": s.value, "bytes": b.value}

    def columns(self, dens, out=None, stream=None):
        import torch
        dens = dens.contiguous()
        if dens.dim() == 1:
            dens = dens[:, None]
        S = int(dens.shape[1])
        odt = torch.float32 if self.mode == MODE_F32_KAHAN else torch.float64
        if out is None:
            out = torch.empty((self.src.shape[0], 12 * self.nside ** 2, S), dtype=odt, device=dens.device)
        _check(_lib.rt_paths_columns(self._h, _dptr(dens), S, F64 if dens.dtype == torch.float64 else F32,
                                     _dptr(out), _stream(stream)))
        return out

    def adjoint(self, grad_out, grad_dens=None, stream=None, ordered=False):
        """Gradient of the densities from the record (accumulated into
        grad_dens); ordered=True sums each leaf in the record's order, the same
        bits on every run (the first such call sorts the record by leaf)."""
        import torch
        gdt = torch.float32 if self.mode == MODE_F32_KAHAN else torch.float64
        grad_out = grad_out.to(gdt).contiguous()
        S = int(grad_out.shape[-1])
        if grad_dens is None:
            grad_dens = torch.zeros((self.tree.n_leaves, S), dtype=torch.float64, device=grad_out.device)
        fn = _lib.rt_paths_adjoint_ordered if ordered else _lib.rt_paths_adjoint
        _check(fn(self._h, _dptr(grad_out), S, _dptr(grad_dens), _stream(stream)))
        return grad_dens

    def close(self):
        if getattr(self, "_h", None):
            _lib.rt_destroy_paths(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace_columns_adjoint(tree: Octree, src, nside: int, grad_out, mode="f32k", grad_dens=None,
                          stream=None, path_policy: int = 0):
    """grad_dens[j,k] += sum over rays of grad_out[s,q,k] * ds(s,q,j) (float64).
    path_policy: 0 automatic (the atomic-free leaf gather where the geometry
    allows it, else the scatter), 1 scatter, 2 scatter from a recorded path,
    3 deterministic (the leaf gather, else an ordered sum over a record)."""
    import torch
    m = _mode(mode)
    src = _check_src(src)
    gdt = torch.float32 if m == MODE_F32_KAHAN else torch.float64
    grad_out = grad_out.to(gdt).contiguous()
    S = int(grad_out.shape[-1])
    if grad_dens is None:
        grad_dens = torch.zeros((tree.n_leaves, S), dtype=torch.float64, device=src.device)
    _check(_lib.rt_trace_columns_adjoint(tree.handle, _dptr(src), int(src.shape[0]), int(nside),
                                         _dptr(grad_out), S, m, _dptr(grad_dens), int(path_policy),
                                         _stream(stream)))
    return grad_dens


def _cloud_descs(clouds, mode: int, outputs=None):
    """Descriptors of (tree, src, nside, dens) clouds, their (new or given)
    outputs and the tensors that must stay alive while they are used."""
    import torch
    odt = torch.float32 if mode == MODE_F32_KAHAN else torch.float64
    descs = (CloudDesc * len(clouds))()
    keep, outs = [], []
    for i, (tree, src, nside, dens) in enumerate(clouds):
        src = _check_src(src)
        dens = dens.contiguous()
        if dens.dim() == 1:
            dens = dens[:, None]
        shape = (src.shape[0], 12 * nside * nside, dens.shape[1])
        out = outputs[i] if outputs is not None else torch.empty(shape, dtype=odt, device=src.device)
        if out.dtype != odt or tuple(out.shape) != shape or not out.is_contiguous():
            raise ValueError(f"output {i} has the wrong dtype, shape or layout")
        keep += [tree, src, dens]
        outs.append(out)
        descs[i] = CloudDesc(tree.handle.value, src.data_ptr(), src.shape[0], nside, dens.shape[1],
                             dens.data_ptr(), F64 if dens.dtype == torch.float64 else F32, 0, out.data_ptr())
    return descs, outs, keep


def trace_batched(clouds, mode="f32k", outputs=None, stream=None):
    """All clouds [(tree, src, nside, dens)] in one persistent launch replayed
    as a CUDA graph (rt_trace_batched; the batch is kept and replayed while the
    same clouds and outputs come back).  Returns the outputs."""
    m = _mode(mode)
    descs, outs, _keep = _cloud_descs(clouds, m, outputs)
    _check(_lib.rt_trace_batched(descs, len(clouds), m, _stream(stream)))
    return outs


def autotune(clouds, mode="f32k", cache_json=None):
    """Tunes and applies the batched launch shape for these clouds (rt_autotune)."""
    m = _mode(mode)
    descs, _outs, _keep = _cloud_descs(clouds, m)
    _check(_lib.rt_autotune(descs, len(clouds), m, cache_json.encode() if cache_json else None))


class Batch:
    """Many clouds traced in one persistent launch, replayed as a CUDA graph.
    clouds: sequence of (tree, src, nside, dens); outputs are allocated here
    (float32 for F32-Kahan, float64 for FP64) and returned by .outputs."""

    def __init__(self, clouds, mode="f32k"):
        import torch
        self.mode = _mode(mode)
        odt = torch.float32 if self.mode == MODE_F32_KAHAN else torch.float64
        self._keep, self.outputs = [], []
        descs = (CloudDesc * len(clouds))()
        for i, (tree, src, nside, dens) in enumerate(clouds):
            src = _check_src(src)
            dens = dens.contiguous()
            if dens.dim() == 1:
                dens = dens[:, None]
            out = torch.empty((src.shape[0], 12 * nside * nside, dens.shape[1]), dtype=odt, device=src.device)
            self._keep += [tree, src, dens]
            self.outputs.append(out)
            descs[i] = CloudDesc(tree.handle.value, src.data_ptr(), src.shape[0], nside, dens.shape[1],
                                 dens.data_ptr(), F64 if dens.dtype == torch.float64 else F32, 0,
                                 out.data_ptr())
        h = C.c_void_p()
        _check(_lib.rt_batch_create(descs, len(clouds), self.mode, C.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(_lib.rt_batch_launch(self._h, _stream(stream)))
        return self.outputs

    def stats(self, stream=None) -> dict:
        s = Stats()
        _check(_lib.rt_batch_stats(self._h, C.byref(s), _stream(stream)))
        return {f: getattr(s, f) for f, _ in Stats._fields_ if f != "reserved"}

    def reset_stats(self, stream=None):
        _check(_lib.rt_batch_reset_stats(self._h, _stream(stream)))

    def autotune(self, cache_json=None, stream=None):
        """Times launch shapes and applies the best; returns ((threads,
        blocks_per_sm, groups_per_pop), segments/s)."""
        best = (C.c_int * 3)()
        rate = C.c_double()
        _check(_lib.rt_batch_autotune(self._h, cache_json.encode() if cache_json else None, C.byref(best),
                                      C.byref(rate), _stream(stream)))
        return tuple(best), rate.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.rt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


try:
    import torch as _torch

    class Columns(_torch.autograd.Function):
        """Differentiable columns: forward = trace_columns, backward = the
        adjoint trace (gradient with respect to the per-leaf densities).  With
        paths (a Paths record of the same tree, sources, nside and mode), both
        are evaluated from the record without walking: the same bits as the
        walk, worth it when the geometry is reused for several steps."""

        @staticmethod
        def forward(ctx, dens, tree, src, nside, mode="f32k", paths=None):
            ctx.tree, ctx.nside, ctx.mode, ctx.paths = tree, nside, mode, paths
            ctx.save_for_backward(src)
            ctx.dens_dtype = dens.dtype
            if paths is not None:
                return paths.columns(dens.detach())
            return trace_columns(tree, src, nside, dens.detach(), mode)

        @staticmethod
        def backward(ctx, g):
            (src,) = ctx.saved_tensors
            if ctx.paths is not None:
                gd = ctx.paths.adjoint(g)
            else:
                gd = trace_columns_adjoint(ctx.tree, src, ctx.nside, g, ctx.mode)
            return gd.to(ctx.dens_dtype), None, None, None, None, None
except ImportError:  # pragma: no cover - torch is required for device memory
    Columns = None
