"""Thin ctypes binding of libwr (include/wr.h), same names as the C ABI.

Argument marshalling only: every step of the rank path runs in libwr's CUDA
kernels.  Device pointers may be given as integers or as objects with a
data_ptr() method (for example torch tensors on the context's device).
Errors raise WrError with the library's status and message.  There is no
fallback: if libwr.so is missing the import of this module fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwr.so")

WR_OK, WR_EINVAL, WR_ENOMEM, WR_EDEVICE, WR_ETIMEDOUT = 0, -1, -2, -3, -4
WR_ENOTPRIME, WR_EOVERFLOW, WR_EPROBFAIL, WR_EBUSY = -5, -6, -7, -8
WR_PROJ_GENERIC, WR_PROJ_SYMMETRIC = 0, 1
WR_SIDE_AUTO, WR_SIDE_COLS, WR_SIDE_ROWS = -1, 0, 1
WR_WANT_SEQUENCE, WR_WANT_GENERATOR = 1, 2


class WrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("wr status %d: %s" % (status, message))
        self.status = status
        self.message = message


class wr_params(ctypes.Structure):
    _fields_ = [("prime", ctypes.c_uint32), ("m", ctypes.c_uint32), ("n", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("projection", ctypes.c_int32), ("side", ctypes.c_int32),
                ("seq_len", ctypes.c_uint64), ("want", ctypes.c_uint32)]


class wr_csr_io(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("out_rows", ctypes.c_int64),
                ("out_cols", ctypes.c_int64), ("rank_offset", ctypes.c_int64), ("out_rowptr", ctypes.c_void_p),
                ("out_colidx", ctypes.c_void_p), ("out_vals", ctypes.c_void_p), ("out_row_of", ctypes.c_void_p),
                ("out_col_of", ctypes.c_void_p)]


class wr_timings(ctypes.Structure):
    _fields_ = [("setup_ms", ctypes.c_double), ("sequence_ms", ctypes.c_double),
                ("sigma_ms", ctypes.c_double), ("readout_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("spmm_ms", ctypes.c_double),
                ("spmm_launches", ctypes.c_int64), ("spmm_bytes", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("sigma_window_ms", ctypes.c_double),
                ("sigma_local_ms", ctypes.c_double), ("sigma_apply_ms", ctypes.c_double),
                ("sigma_tail_ms", ctypes.c_double), ("sequence_terms", ctypes.c_int64),
                ("sigma_product_ms", ctypes.c_double)]


class wr_server_cfg(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("hbm_budget", ctypes.c_uint64), ("queue_cap", ctypes.c_int32)]


class wr_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("throughput_rps", ctypes.c_double), ("max_resident", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64)]


if not os.path.exists(LIB_PATH):
    raise ImportError("libwr.so is not built (run __graft_entry__.build()); there is no fallback")
_lib = ctypes.CDLL(LIB_PATH)

vp, i64, u64, u32, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
P = ctypes.POINTER
_sig = {
    "wr_create": ([P(vp), ctypes.c_int, vp], ctypes.c_int),
    "wr_destroy": ([vp], None),
    "wr_last_error": ([], ctypes.c_char_p),
    "wr_set_profiling": ([vp, ctypes.c_int], ctypes.c_int),
    "wr_last_timings": ([vp, P(wr_timings)], ctypes.c_int),
    "wr_set_sigma_chunk": ([vp, i32], ctypes.c_int),
    "wr_set_sigma_leaf": ([vp, i64], ctypes.c_int),
    "wr_set_autotune": ([vp, i32], ctypes.c_int),
    "wr_set_allocator": ([vp, vp, vp, vp], ctypes.c_int),
    "wr_set_lane_width": ([vp, i32], ctypes.c_int),
    "wr_set_paired_projection": ([vp, i32], ctypes.c_int),
    "wr_set_tensor_projection": ([vp, i32], ctypes.c_int),
    "wr_set_column_slabs": ([vp, i64], ctypes.c_int),
    "wr_sequence_state_device": ([vp, vp, P(wr_params), vp, u64, i64, vp, vp, P(i64), P(i32)], ctypes.c_int),
    "wr_gram_device": ([vp, u32, i64, u32, u32, vp, i32, i32, vp, vp], ctypes.c_int),
    "wr_probe_mma": ([vp, i64, i32, vp, P(ctypes.c_double)], ctypes.c_int),
    "wr_polymat_mul_device": ([vp, u32, vp, i64, vp, i64, u32, u32, u32, i64, i64, vp], ctypes.c_int),
    "wr_set_projection_overlap": ([vp, i32], ctypes.c_int),
    "wr_set_pipeline": ([vp, i32], ctypes.c_int),
    "wr_set_early_termination": ([vp, i64], ctypes.c_int),
    "wr_set_chain_reduction": ([vp, i32], ctypes.c_int),
    "wr_set_locality_order": ([vp, i32], ctypes.c_int),
    "wr_locality_order_csr": ([i64, i64, vp, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
    "wr_chain_reduce_complex": ([i32, vp], ctypes.c_int),
    "wr_matrix_reduction": ([vp, P(i64), P(i64), P(i64)], ctypes.c_int),
    "wr_chain_reduce_csr": ([i64, i64, vp, vp, vp, P(i64), P(i64), vp, vp, vp, vp, vp, P(i64)], ctypes.c_int),
    "wr_matrix_load_csr": ([vp, i64, i64, vp, vp, vp, P(vp)], ctypes.c_int),
    "wr_matrix_load_csr_device": ([vp, i64, i64, i64, vp, vp, vp, P(vp)], ctypes.c_int),
    "wr_matrix_info": ([vp, P(i64), P(i64), P(i64), P(i64), P(i64)], ctypes.c_int),
    "wr_matrix_free": ([vp], None),
    "wr_rank": ([vp, vp, P(wr_params), P(vp)], ctypes.c_int),
    "wr_rank_batch": ([vp, ctypes.c_size_t, P(vp), P(wr_params), P(vp)], ctypes.c_int),
    "wr_set_batch_slots": ([vp, i32], ctypes.c_int),
    "wr_set_batch_fusion": ([vp, i32], ctypes.c_int),
    "wr_rank_device_bytes": ([vp, vp, P(wr_params), P(u64)], ctypes.c_int),
    "wr_result_rank": ([vp], u64),
    "wr_result_info": ([vp, P(i64), P(i64), P(i64), P(i64)], ctypes.c_int),
    "wr_result_sequence": ([vp, vp, ctypes.c_size_t], ctypes.c_int),
    "wr_result_generator": ([vp, vp, ctypes.c_size_t, vp], ctypes.c_int),
    "wr_result_free": ([vp], None),
    "wr_blackbox_apply_device": ([vp, vp, P(wr_params), vp, vp, i64], ctypes.c_int),
    "wr_blackbox_apply_device_noalloc": ([vp, vp, P(wr_params), vp, vp, i64], ctypes.c_int),
    "wr_sequence_device": ([vp, vp, P(wr_params), vp, u64], ctypes.c_int),
    "wr_sequence_slab_device": ([vp, vp, P(wr_params), u32, u32, vp, u64], ctypes.c_int),
    "wr_sigma_basis_device": ([vp, vp, u64, u32, u32, u32, vp, vp, i64], ctypes.c_int),
    "wr_det_valuation_device": ([vp, vp, i64, i64, u32, P(i64)], ctypes.c_int),
    "wr_server_start": ([vp, P(wr_server_cfg), P(vp)], ctypes.c_int),
    "wr_submit": ([vp, vp, P(wr_params), P(u64)], ctypes.c_int),
    "wr_wait": ([vp, u64, u32, P(vp)], ctypes.c_int),
    "wr_server_stats": ([vp, P(wr_stats)], ctypes.c_int),
    "wr_server_stop": ([vp], None),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def _check(st: int):
    if st != WR_OK:
        raise WrError(st, _lib.wr_last_error().decode(errors="replace"))


def _dptr(x) -> int:
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x)


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def make_params(prime: int, m: int, n: int, seed: int, projection: int = WR_PROJ_GENERIC,
                side: int = WR_SIDE_AUTO, seq_len: int = 0, want: int = 0) -> wr_params:
    return wr_params(prime, m, n, seed & 0xFFFFFFFFFFFFFFFF, projection, side, seq_len, want)


# ------------------------------------------------------------------ context

def wr_create(device: int = 0, stream=None) -> int:
    h = vp()
    _check(_lib.wr_create(ctypes.byref(h), device, vp(_dptr(stream) if stream is not None else None)))
    return h.value


def wr_destroy(ctx: int) -> None:
    _lib.wr_destroy(vp(ctx))


def wr_last_error() -> str:
    return _lib.wr_last_error().decode(errors="replace")


def wr_set_profiling(ctx: int, on: bool) -> None:
    _check(_lib.wr_set_profiling(vp(ctx), 1 if on else 0))


def wr_last_timings(ctx: int) -> dict:
    t = wr_timings()
    _check(_lib.wr_last_timings(vp(ctx), ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in wr_timings._fields_}


# ------------------------------------------------------------------ matrices

def wr_matrix_load_csr(ctx: int, rows: int, cols: int, rowptr, colidx, vals) -> int:
    rp = _np(rowptr, np.int64)
    ci = _np(colidx, np.int32)
    va = _np(vals, np.int32)
    h = vp()
    _check(_lib.wr_matrix_load_csr(vp(ctx), rows, cols, rp.ctypes.data, ci.ctypes.data, va.ctypes.data,
                                   ctypes.byref(h)))
    return h.value


def wr_matrix_load_csr_device(ctx: int, rows: int, cols: int, nnz: int, d_rowptr, d_colidx, d_vals) -> int:
    h = vp()
    _check(_lib.wr_matrix_load_csr_device(vp(ctx), rows, cols, nnz, vp(_dptr(d_rowptr)), vp(_dptr(d_colidx)),
                                          vp(_dptr(d_vals)), ctypes.byref(h)))
    return h.value


def wr_matrix_info(mat: int) -> dict:
    v = [i64() for _ in range(5)]
    _check(_lib.wr_matrix_info(vp(mat), *[ctypes.byref(x) for x in v]))
    return dict(zip(["rows", "cols", "nnz", "slots_a", "slots_at"], [x.value for x in v]))


def wr_matrix_free(mat: int) -> None:
    _lib.wr_matrix_free(vp(mat))


# ------------------------------------------------------------------ rank

def wr_rank(ctx: int, mat: int, params: wr_params) -> int:
    h = vp()
    _check(_lib.wr_rank(vp(ctx), vp(mat), ctypes.byref(params), ctypes.byref(h)))
    return h.value


def wr_rank_batch(ctx: int, mats: Sequence[int], params: Sequence[wr_params]) -> list:
    n = len(mats)
    marr = (vp * n)(*[vp(m) for m in mats])
    parr = (wr_params * n)(*params)
    outs = (vp * n)()
    _check(_lib.wr_rank_batch(vp(ctx), n, marr, parr, outs))
    return [o for o in outs]


def wr_set_sigma_chunk(ctx: int, orders: int) -> None:
    _check(_lib.wr_set_sigma_chunk(vp(ctx), orders))


def wr_set_sigma_leaf(ctx: int, orders: int) -> None:
    _check(_lib.wr_set_sigma_leaf(vp(ctx), orders))


WR_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
WR_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


def wr_set_allocator(ctx: int, alloc=None, release=None, user=None) -> None:
    """alloc(bytes, stream) -> device pointer (int), release(ptr, bytes, stream):
    Python callables wrapped as the C callbacks (kept alive on the binding),
    or None, None for the default pool."""
    if alloc is None and release is None:
        _check(_lib.wr_set_allocator(vp(ctx), None, None, None))
        _allocators.pop(ctx, None)
        return
    fa = WR_ALLOC_FN(lambda n, s, u: alloc(n, s or 0) or None) if alloc is not None else None
    ff = WR_FREE_FN(lambda p, n, s, u: release(p, n, s or 0)) if release is not None else None
    _check(_lib.wr_set_allocator(vp(ctx), ctypes.cast(fa, vp) if fa else None,
                                 ctypes.cast(ff, vp) if ff else None, None))
    _allocators[ctx] = (fa, ff)


_allocators = {}


def wr_set_autotune(ctx: int, on: bool) -> None:
    _check(_lib.wr_set_autotune(vp(ctx), 1 if on else 0))


def wr_set_lane_width(ctx: int, residues: int) -> None:
    _check(_lib.wr_set_lane_width(vp(ctx), residues))


def wr_set_column_slabs(ctx: int, nbytes: int) -> None:
    _check(_lib.wr_set_column_slabs(vp(ctx), nbytes))


def wr_set_tensor_projection(ctx: int, mode: int) -> None:
    _check(_lib.wr_set_tensor_projection(vp(ctx), mode))


def wr_set_paired_projection(ctx: int, on: bool) -> None:
    _check(_lib.wr_set_paired_projection(vp(ctx), 1 if on else 0))


def wr_set_projection_overlap(ctx: int, on: bool) -> None:
    _check(_lib.wr_set_projection_overlap(vp(ctx), 1 if on else 0))


def wr_set_pipeline(ctx: int, mode: int) -> None:
    """0 off, 1 (True) the sequence's stream first, 2 the sigma-basis's first."""
    _check(_lib.wr_set_pipeline(vp(ctx), int(mode)))


def wr_set_early_termination(ctx: int, orders: int) -> None:
    _check(_lib.wr_set_early_termination(vp(ctx), orders))


def wr_set_chain_reduction(ctx: int, on: bool) -> None:
    _check(_lib.wr_set_chain_reduction(vp(ctx), 1 if on else 0))


def wr_set_locality_order(ctx: int, on: bool) -> None:
    _check(_lib.wr_set_locality_order(vp(ctx), 1 if on else 0))


def wr_locality_order_csr(rows: int, cols: int, rowptr, colidx, vals):
    """Host locality order (no device needed): returns (rowptr, colidx, vals,
    row_of, col_of) of the renumbered CSR."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.int32)
    nnz = int(rowptr[rows])
    orp = np.zeros(rows + 1, dtype=np.int64)
    oci = np.zeros(max(nnz, 1), dtype=np.int32)
    ova = np.zeros(max(nnz, 1), dtype=np.int32)
    rof = np.zeros(max(rows, 1), dtype=np.int32)
    cof = np.zeros(max(cols, 1), dtype=np.int32)
    _check(_lib.wr_locality_order_csr(rows, cols, vp(rowptr.ctypes.data), vp(colidx.ctypes.data),
                                      vp(vals.ctypes.data), vp(orp.ctypes.data), vp(oci.ctypes.data),
                                      vp(ova.ctypes.data), vp(rof.ctypes.data), vp(cof.ctypes.data)))
    return orp, oci[:nnz].copy(), ova[:nnz].copy(), rof[:rows].copy(), cof[:cols].copy()


def wr_chain_reduce_complex(mats):
    """Host chain reduction along a complex (no device needed).  mats: list of
    (rows, cols, rowptr, colidx, vals) with mats[i] mats[i+1] = 0.  Returns a
    list of (rows, cols, rowptr, colidx, vals, row_of, col_of, rank_offset)."""
    k = len(mats)
    arr = (wr_csr_io * max(k, 1))()
    keep = []
    for i, (rows, cols, rowptr, colidx, vals) in enumerate(mats):
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.int32)
        nnz = int(rowptr[rows])
        outs = (np.zeros(rows + 1, dtype=np.int64), np.zeros(max(nnz, 1), dtype=np.int32),
                np.zeros(max(nnz, 1), dtype=np.int32), np.zeros(max(rows, 1), dtype=np.int32),
                np.zeros(max(cols, 1), dtype=np.int32))
        keep.append((rowptr, colidx, vals) + outs)
        a = arr[i]
        a.rows, a.cols = rows, cols
        a.rowptr, a.colidx, a.vals = rowptr.ctypes.data, colidx.ctypes.data, vals.ctypes.data
        a.out_rowptr, a.out_colidx, a.out_vals, a.out_row_of, a.out_col_of = [o.ctypes.data for o in outs]
    _check(_lib.wr_chain_reduce_complex(k, ctypes.cast(arr, ctypes.c_void_p)))
    res = []
    for i in range(k):
        a = arr[i]
        orp, oci, ova, rof, cof = keep[i][3:]
        n2 = int(orp[a.out_rows])
        res.append((a.out_rows, a.out_cols, orp[: a.out_rows + 1].copy(), oci[:n2].copy(), ova[:n2].copy(),
                    rof[: a.out_rows].copy(), cof[: a.out_cols].copy(), a.rank_offset))
    return res


def wr_matrix_reduction(mat: int) -> dict:
    a, b, c = i64(), i64(), i64()
    _check(_lib.wr_matrix_reduction(vp(mat), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return dict(rows_in=a.value, cols_in=b.value, rank_offset=c.value)


def wr_chain_reduce_csr(rows: int, cols: int, rowptr, colidx, vals):
    """Host chain reduction (no device needed): returns (rows, cols, rowptr,
    colidx, vals, row_of, col_of, rank_offset) of the reduced CSR, row_of and
    col_of being the kept rows' and columns' input indices."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.int32)
    nnz = int(rowptr[rows])
    orp = np.zeros(rows + 1, dtype=np.int64)
    oci = np.zeros(max(nnz, 1), dtype=np.int32)
    ova = np.zeros(max(nnz, 1), dtype=np.int32)
    rof = np.zeros(max(rows, 1), dtype=np.int32)
    cof = np.zeros(max(cols, 1), dtype=np.int32)
    r, c, off = i64(), i64(), i64()
    _check(_lib.wr_chain_reduce_csr(rows, cols, vp(rowptr.ctypes.data), vp(colidx.ctypes.data),
                                    vp(vals.ctypes.data), ctypes.byref(r), ctypes.byref(c),
                                    vp(orp.ctypes.data), vp(oci.ctypes.data), vp(ova.ctypes.data),
                                    vp(rof.ctypes.data), vp(cof.ctypes.data), ctypes.byref(off)))
    n2 = int(orp[r.value])
    return (r.value, c.value, orp[: r.value + 1].copy(), oci[:n2].copy(), ova[:n2].copy(),
            rof[: r.value].copy(), cof[: c.value].copy(), off.value)


def wr_set_batch_fusion(ctx: int, on: bool) -> None:
    _check(_lib.wr_set_batch_fusion(vp(ctx), 1 if on else 0))


def wr_set_batch_slots(ctx: int, slots: int) -> None:
    _check(_lib.wr_set_batch_slots(vp(ctx), slots))


def wr_rank_device_bytes(ctx: int, mat: int, params: wr_params) -> int:
    b = u64()
    _check(_lib.wr_rank_device_bytes(vp(ctx), vp(mat), ctypes.byref(params), ctypes.byref(b)))
    return b.value


def wr_result_rank(res: int) -> int:
    return int(_lib.wr_result_rank(vp(res)))


def wr_result_info(res: int) -> dict:
    v = [i64() for _ in range(4)]
    _check(_lib.wr_result_info(vp(res), *[ctypes.byref(x) for x in v]))
    return dict(zip(["deg_det", "codeg", "sum_delta", "seq_len"], [x.value for x in v]))


def wr_result_sequence(res: int, m: int, n: int) -> np.ndarray:
    L = wr_result_info(res)["seq_len"]
    out = np.empty(L * m * n, dtype=np.uint32)
    _check(_lib.wr_result_sequence(vp(res), out.ctypes.data, out.size))
    return out.reshape(L, m, n)


def wr_result_generator(res: int, n: int):
    deg = np.empty(n, dtype=np.int32)
    _check(_lib.wr_result_generator(vp(res), None, 0, deg.ctypes.data))
    dmax = int(deg.max()) if n else 0
    coeffs = np.empty((dmax + 1) * n * n, dtype=np.uint32)
    _check(_lib.wr_result_generator(vp(res), coeffs.ctypes.data, coeffs.size, deg.ctypes.data))
    return coeffs.reshape(dmax + 1, n, n), deg


def wr_result_free(res: int) -> None:
    _lib.wr_result_free(vp(res))


# ------------------------------------------------------------------ step-level calls

def wr_blackbox_apply_device(ctx: int, mat: int, params: wr_params, d_in, d_out, width: int) -> None:
    _check(_lib.wr_blackbox_apply_device(vp(ctx), vp(mat), ctypes.byref(params), vp(_dptr(d_in)),
                                         vp(_dptr(d_out)), width))


def wr_blackbox_apply_device_noalloc(ctx: int, mat: int, params: wr_params, d_in, d_out, width: int) -> None:
    """Same as wr_blackbox_apply_device, with no device allocation (fixed
    per-device scratch; see include/wr.h)."""
    _check(_lib.wr_blackbox_apply_device_noalloc(vp(ctx), vp(mat), ctypes.byref(params), vp(_dptr(d_in)),
                                                 vp(_dptr(d_out)), width))


def wr_sequence_device(ctx: int, mat: int, params: wr_params, d_S, L: int) -> None:
    _check(_lib.wr_sequence_device(vp(ctx), vp(mat), ctypes.byref(params), vp(_dptr(d_S)), L))


def wr_sequence_state_device(ctx: int, mat: int, params: wr_params, d_S, L: int, snap_at: int = -1,
                             d_snap=None, d_last=None):
    """Returns (applications, paired)."""
    k, pr = i64(), i32()
    _check(_lib.wr_sequence_state_device(vp(ctx), vp(mat), ctypes.byref(params), vp(_dptr(d_S)), L, snap_at,
                                         vp(_dptr(d_snap)), vp(_dptr(d_last)), ctypes.byref(k), ctypes.byref(pr)))
    return k.value, bool(pr.value)


def wr_gram_device(ctx: int, prime: int, N: int, m: int, n: int, d_t, tstride: int, yoff: int, d_w, d_G) -> None:
    _check(_lib.wr_gram_device(vp(ctx), prime, N, m, n, vp(_dptr(d_t)), tstride, yoff, vp(_dptr(d_w)),
                               vp(_dptr(d_G))))


def wr_polymat_mul_device(ctx: int, prime: int, d_A, na: int, d_B, nb: int, r: int, s: int, t: int, lo: int,
                          hi: int, d_C) -> None:
    _check(_lib.wr_polymat_mul_device(vp(ctx), prime, vp(_dptr(d_A)), na, vp(_dptr(d_B)), nb, r, s, t, lo, hi,
                                      vp(_dptr(d_C))))


def wr_probe_mma(ctx: int, iters: int, blocks: int, d_out=None) -> float:
    """Kernel time in ms of the tensor-core probe (see include/wr.h)."""
    ms = ctypes.c_double()
    _check(_lib.wr_probe_mma(vp(ctx), iters, blocks, vp(_dptr(d_out)), ctypes.byref(ms)))
    return ms.value


def wr_sequence_slab_device(ctx: int, mat: int, params: wr_params, col0: int, ncols: int, d_S, L: int) -> None:
    _check(_lib.wr_sequence_slab_device(vp(ctx), vp(mat), ctypes.byref(params), col0, ncols,
                                        vp(_dptr(d_S)), L))


def wr_sigma_basis_device(ctx: int, d_S, L: int, m: int, n: int, prime: int, d_P, d_deg, Dcap: int) -> None:
    _check(_lib.wr_sigma_basis_device(vp(ctx), vp(_dptr(d_S)), L, m, n, prime, vp(_dptr(d_P)),
                                      vp(_dptr(d_deg)), Dcap))


def wr_det_valuation_device(ctx: int, d_G, n: int, T: int, prime: int) -> int:
    v = i64()
    _check(_lib.wr_det_valuation_device(vp(ctx), vp(_dptr(d_G)), n, T, prime, ctypes.byref(v)))
    return v.value


# ------------------------------------------------------------------ serving

def wr_server_start(ctx: int, max_slots: int = 8, hbm_budget: int = 0, queue_cap: int = 0) -> int:
    cfg = wr_server_cfg(max_slots, hbm_budget, queue_cap)
    h = vp()
    _check(_lib.wr_server_start(vp(ctx), ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def wr_submit(srv: int, mat: int, params: wr_params) -> int:
    t = u64()
    _check(_lib.wr_submit(vp(srv), vp(mat), ctypes.byref(params), ctypes.byref(t)))
    return t.value


def wr_wait(srv: int, ticket: int, timeout_ms: int) -> int:
    h = vp()
    _check(_lib.wr_wait(vp(srv), ticket, timeout_ms, ctypes.byref(h)))
    return h.value


def wr_server_stats(srv: int) -> dict:
    s = wr_stats()
    _check(_lib.wr_server_stats(vp(srv), ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in wr_stats._fields_}


def wr_server_stop(srv: int) -> None:
    _lib.wr_server_stop(vp(srv))
