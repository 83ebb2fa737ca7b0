"""Thin ctypes binding of the C ABI in include/pw.h (argument marshalling only).

Every numerical step runs in the CUDA library libpwgb300.so.  Importing this
module fails loudly if the library has not been built: there is no CPU
fallback.  Device buffers are torch CUDA tensors (complex128), passed by
data_ptr() together with the current torch stream.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpwgb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ct.CDLL(LIB_PATH)

PW_OK, PW_ERR_ARG, PW_ERR_OOM, PW_ERR_CUDA, PW_ERR_CHOL, PW_ERR_NOCONV, PW_ERR_TIMEOUT, \
    PW_ERR_BUSY, PW_ERR_NUMERIC = 0, -1, -2, -3, -4, -5, -6, -7, -8
PW_FP64, PW_MIXED = 0, 1
_PREC = {"fp64": PW_FP64, "mixed": PW_MIXED, PW_FP64: PW_FP64, PW_MIXED: PW_MIXED}


class PwError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {pw_strerror(status)} ({status})")


class pw_cell_desc(ct.Structure):
    _fields_ = [("lattice", ct.c_double * 9), ("natom", ct.c_int),
                ("tau", ct.POINTER(ct.c_double)), ("vdepth", ct.POINTER(ct.c_double)),
                ("vwidth", ct.c_double), ("pwidth", ct.c_double),
                ("dkb", ct.POINTER(ct.c_double)), ("ecut", ct.c_double),
                ("grid", ct.c_int * 3), ("precision", ct.c_int)]


class pw_solve_opts(ct.Structure):
    _fields_ = [("nbands", ct.c_int), ("tol", ct.c_double), ("maxit", ct.c_int),
                ("seed", ct.c_uint64), ("x0", ct.c_void_p), ("precision", ct.c_int),
                ("chunk_rows", ct.c_int), ("h_blocks", ct.c_int)]


class pw_step_report(ct.Structure):
    _fields_ = [("iter", ct.c_int), ("nactive", ct.c_int), ("dropped_p", ct.c_int),
                ("nsub", ct.c_int), ("max_resid", ct.c_double), ("ms", ct.c_double),
                ("ms_resid", ct.c_double), ("ms_hpsi", ct.c_double), ("ms_gram", ct.c_double),
                ("ms_rr", ct.c_double), ("ms_rot", ct.c_double),
                ("ms_rr_part", ct.c_double * 5), ("hpsi_cols", ct.c_int)]


class pw_request(ct.Structure):
    _fields_ = [("species", ct.c_int), ("ncell", ct.c_int), ("ecut", ct.c_double),
                ("nbands", ct.c_int), ("seed", ct.c_uint64), ("t_arrival", ct.c_double),
                ("tol", ct.c_double), ("maxit", ct.c_int)]


class pw_result(ct.Structure):
    _fields_ = [("eig", ct.POINTER(ct.c_double)), ("status", ct.c_int), ("iters", ct.c_int),
                ("npw", ct.c_int), ("max_resid", ct.c_double), ("orth_err", ct.c_double),
                ("t_admit", ct.c_double), ("t_done", ct.c_double), ("latency", ct.c_double),
                ("hbm_bytes", ct.c_size_t)]


class pw_serve_opts(ct.Structure):
    _fields_ = [("max_slots", ct.c_int), ("hbm_budget", ct.c_size_t), ("precision", ct.c_int),
                ("time_scale", ct.c_double), ("autotune", ct.c_int), ("batch_fft", ct.c_int),
                ("batch_window_us", ct.c_double)]


class pw_solve_report(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("fp64_iters", ct.c_int), ("max_resid", ct.c_double), ("orth_err", ct.c_double),
                ("seconds", ct.c_double), ("device_bytes", ct.c_size_t)]


class _Fn:
    """Resolves a library symbol on first call (with its C signature)."""

    def __init__(self, name, res, args):
        self.name, self.res, self.args, self.f = name, res, args, None

    def __call__(self, *a):
        if self.f is None:
            f = getattr(_lib, self.name)
            f.restype, f.argtypes = self.res, self.args
            self.f = f
        return self.f(*a)


def _sig(name, res, args):
    return _Fn(name, res, args)


_vp = ct.c_void_p
_setup = _sig("pw_setup_cell", ct.c_int, [ct.POINTER(pw_cell_desc), _vp, ct.POINTER(_vp)])
_info = _sig("pw_cell_info", ct.c_int, [_vp, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                        ct.POINTER(ct.POINTER(ct.c_int))])
_sizes = _sig("pw_cell_sizes", ct.c_int, [_vp, ct.POINTER(ct.c_int), ct.POINTER(ct.c_size_t)])
_setprec = _sig("pw_cell_set_precision", ct.c_int, [_vp, ct.c_int])
_apply = _sig("pw_apply_H", ct.c_int, [_vp, _vp, ct.c_int, ct.c_int, _vp, _vp])
_destroy = _sig("pw_destroy_cell", None, [_vp])
_strerror = _sig("pw_strerror", ct.c_char_p, [ct.c_int])
_screate = _sig("pw_solver_create", ct.c_int, [_vp, ct.POINTER(pw_solve_opts), _vp, ct.POINTER(_vp)])
_sstep = _sig("pw_subspace_step", ct.c_int, [_vp, _vp, ct.POINTER(pw_step_report)])
_seigs = _sig("pw_solver_eigs", ct.c_int, [_vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)])
_sblock = _sig("pw_solver_block", ct.c_int, [_vp, _vp, ct.c_int])
_sdestroy = _sig("pw_solver_destroy", None, [_vp])
_eigsolve = _sig("pw_eigsolve", ct.c_int, [_vp, ct.POINTER(pw_solve_opts), ct.POINTER(ct.c_double),
                                            _vp, ct.c_int, ct.POINTER(pw_solve_report), _vp])


_heev = _sig("pw_heev", ct.c_int, [ct.c_int, ct.c_int, _vp, _vp, _vp, _vp])


def pw_heev(A, nb, stream=None):
    """Lowest nb eigenpairs of a Hermitian CUDA complex128 (n, n) tensor (column-major
    copy is made).  Returns (w (n,), Y (n, nb)) as CUDA tensors."""
    import torch
    n = A.shape[0]
    a = A.t().contiguous().t().clone()       # column-major working copy
    if a.stride(0) != 1:
        a = a.t().contiguous().t()
    w = torch.empty(n, dtype=torch.float64, device=A.device)
    Y = torch.empty((nb, n), dtype=torch.complex128, device=A.device).T
    _check(_heev(n, nb, _dptr(a), _dptr(w), _dptr(Y), _stream(stream)), "pw_heev")
    return w, Y


_zgemm_tc = _sig("pw_zgemm_tc", ct.c_int, [ct.c_char, ct.c_int, ct.c_int, ct.c_int, _vp, ct.c_int,
                                            _vp, ct.c_int, ct.c_double, _vp, ct.c_int, _vp])


def pw_zgemm_tc(opA, A, B, C=None, beta=0.0, stream=None):
    """C = A^H B (opA 'C') or A B (opA 'N') with split-FP16 tensor-core arithmetic.
    A, B, C: column-major CUDA complex128 tensors (stride(0) == 1)."""
    import torch
    if opA == "C":
        k, m = A.shape
    else:
        m, k = A.shape
    n = B.shape[1]
    if C is None:
        C = torch.zeros((n, m), dtype=torch.complex128, device=A.device).T
    for t in (A, B, C):
        assert t.stride(0) == 1
    _check(_zgemm_tc(opA.encode(), m, n, k, _dptr(A), A.stride(1), _dptr(B), B.stride(1),
                     float(beta), _dptr(C), C.stride(1), _stream(stream)), "pw_zgemm_tc")
    return C


_zgemm_f64tc = _sig("pw_zgemm_f64tc", ct.c_int, [ct.c_char, ct.c_char, ct.c_int, ct.c_int, ct.c_int,
                                                  ct.POINTER(ct.c_double), _vp, ct.c_int, _vp, ct.c_int,
                                                  ct.POINTER(ct.c_double), _vp, ct.c_int, _vp])


def pw_zgemm_f64tc(opA, opB, A, B, C=None, alpha=1.0, beta=0.0, stream=None):
    """C = alpha op(A) op(B) + beta C, FP64-accurate on the FP16 tensor cores.
    A, B, C: column-major CUDA complex128 tensors (stride(0) == 1)."""
    import torch
    m, k = (A.shape if opA == "N" else A.shape[::-1])
    n = B.shape[1] if opB == "N" else B.shape[0]
    if C is None:
        C = torch.zeros((n, m), dtype=torch.complex128, device=A.device).T
    for t in (A, B, C):
        assert t.stride(0) == 1
    a = (ct.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    b = (ct.c_double * 2)(complex(beta).real, complex(beta).imag)
    ld = lambda t: max(t.stride(1), t.shape[0], 1)
    _check(_zgemm_f64tc(opA.encode(), opB.encode(), m, n, k, a, _dptr(A), ld(A), _dptr(B), ld(B), b,
                        _dptr(C), ld(C), _stream(stream)), "pw_zgemm_f64tc")
    return C


_dense_products = _sig("pw_dense_products", ct.c_int, [ct.c_int])


def pw_dense_products(mode):
    """1: large products of the FP64 Rayleigh-Ritz on the tensor cores (FP64-accurate); 0: FP64 pipe."""
    _check(_dense_products(int(mode)), "pw_dense_products")


_dense_graphs = _sig("pw_dense_graphs", ct.c_int, [ct.c_int])


def pw_dense_graphs(on):
    """1: capture and replay the eigensolver stages as CUDA graphs (non-default streams); 0: direct launches."""
    _check(_dense_graphs(int(on)), "pw_dense_graphs")


_hh_panels = _sig("pw_householder_panels", ct.c_int, [ct.c_int])


def pw_householder_panels(mode):
    """0 (default): chained kernels per Householder column, Hermitian products of
    large panels on the tensor cores; 1: one cooperative launch per panel (FP64
    products); 2: chained kernels, every Hermitian product on the FP64 pipe;
    3: as 0 with each tensor-core panel in one cooperative launch."""
    _check(_hh_panels(int(mode)), "pw_householder_panels")


_launches = _sig("pw_kernel_launches", ct.c_uint64, [])


def pw_kernel_launches() -> int:
    return int(_launches())


_serve = _sig("pw_serve", ct.c_int, [ct.POINTER(pw_serve_opts), ct.POINTER(pw_request), ct.c_int,
                                      ct.POINTER(pw_result)])
_footprint = _sig("pw_request_footprint", ct.c_size_t, [ct.POINTER(pw_request), ct.c_int])


def _mkreq(r):
    q = pw_request()
    q.species = {"Si": 0, "C": 1, 0: 0, 1: 1}[r["species"]]
    q.ncell, q.ecut, q.nbands = int(r["n"]), float(r["ecut"]), int(r["nbands"])
    q.seed, q.t_arrival = int(r["seed"]), float(r.get("t_arrival", 0.0))
    q.tol, q.maxit = float(r.get("tol", 0.0)), int(r.get("maxit", 0))
    return q


def pw_request_footprint(r, precision="fp64"):
    return int(_footprint(ct.byref(_mkreq(r)), _PREC[precision]))


_batch_stats = _sig("pw_fft_batch_stats", None, [ct.POINTER(ct.c_uint64), ct.POINTER(ct.c_uint64)])


def pw_fft_batch_stats():
    """(launches, band blocks) of the serving loop's cross-request FFT launches so far."""
    a, b = ct.c_uint64(), ct.c_uint64()
    _batch_stats(ct.byref(a), ct.byref(b))
    return a.value, b.value


def pw_serve(requests, max_slots=4, hbm_budget=0, precision="fp64", time_scale=1.0, autotune=False,
             batch_fft=True, batch_window_us=0.0):
    """Serve a list of request dicts (species, n, ecut, nbands, seed, t_arrival[, tol, maxit]).
    Returns a list of dicts with eig (numpy), status, iters, timings."""
    n = len(requests)
    reqs = (pw_request * max(n, 1))(*[_mkreq(r) for r in requests])
    eigs = [np.zeros(int(r["nbands"])) for r in requests]
    res = (pw_result * max(n, 1))()
    for i in range(n):
        res[i].eig = eigs[i].ctypes.data_as(ct.POINTER(ct.c_double))
    o = pw_serve_opts()
    o.max_slots, o.hbm_budget, o.precision, o.time_scale = int(max_slots), int(hbm_budget), \
        _PREC[precision], float(time_scale)
    o.autotune = 1 if autotune else 0
    o.batch_fft = 1 if batch_fft else 0
    o.batch_window_us = float(batch_window_us)
    _check(_serve(ct.byref(o), reqs, n, res), "pw_serve")
    out = []
    for i in range(n):
        r = res[i]
        out.append(dict(eig=eigs[i], status=r.status, iters=r.iters, npw=r.npw,
                        max_resid=r.max_resid, orth_err=r.orth_err, t_admit=r.t_admit,
                        t_done=r.t_done, latency=r.latency, hbm_bytes=r.hbm_bytes))
    return out


def pw_strerror(status: int) -> str:
    return _strerror(int(status)).decode()


def _check(status: int, what: str):
    if status != PW_OK:
        raise PwError(status, what)


def _stream(stream):
    if stream is not None:
        return ct.c_void_p(int(stream))
    import torch
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t):
    return ct.c_void_p(t.data_ptr())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def pw_setup_cell(L, tau, depth, dkb, ecut, vwidth=1.2, pwidth=1.2, grid=None,
                  precision="fp64", stream=None):
    """Build a cell on the current device.  L: scalar (cubic) or 3 lengths."""
    Ls = np.broadcast_to(np.asarray(L, float), (3,))
    tau, depth, dkb = _f64(tau).reshape(-1, 3), _f64(depth).reshape(-1), _f64(dkb).reshape(-1, 4)
    d = pw_cell_desc()
    lat = [0.0] * 9
    lat[0], lat[4], lat[8] = float(Ls[0]), float(Ls[1]), float(Ls[2])
    d.lattice = (ct.c_double * 9)(*lat)
    d.natom = tau.shape[0]
    keep = (tau, depth, dkb)
    d.tau = keep[0].ctypes.data_as(ct.POINTER(ct.c_double))
    d.vdepth = keep[1].ctypes.data_as(ct.POINTER(ct.c_double))
    d.dkb = keep[2].ctypes.data_as(ct.POINTER(ct.c_double))
    d.vwidth, d.pwidth, d.ecut = float(vwidth), float(pwidth), float(ecut)
    d.grid = (ct.c_int * 3)(*(grid if grid is not None else (0, 0, 0)))
    d.precision = _PREC[precision]
    h = ct.c_void_p()
    _check(_setup(ct.byref(d), _stream(stream), ct.byref(h)), "pw_setup_cell")
    return h


def pw_cell_info(cell):
    npw = ct.c_int()
    grid = (ct.c_int * 3)()
    mp = ct.POINTER(ct.c_int)()
    _check(_info(cell, ct.byref(npw), grid, ct.byref(mp)), "pw_cell_info")
    m = np.ctypeslib.as_array(mp, shape=(npw.value * 3,)).reshape(-1, 3).astype(np.int64)
    return npw.value, tuple(grid), m


def pw_cell_sizes(cell):
    nproj = ct.c_int()
    nbytes = ct.c_size_t()
    _check(_sizes(cell, ct.byref(nproj), ct.byref(nbytes)), "pw_cell_sizes")
    return nproj.value, nbytes.value


def pw_cell_set_precision(cell, precision):
    _check(_setprec(cell, _PREC[precision]), "pw_cell_set_precision")


def pw_apply_H(cell, psi, hpsi, stream=None):
    """hpsi <- H psi; psi, hpsi: CUDA complex128 tensors (npw, nb), column-major."""
    assert psi.dtype == hpsi.dtype and psi.is_cuda and hpsi.is_cuda
    npw, nb = psi.shape
    ld = psi.stride(1) if nb > 1 else npw
    assert psi.stride(0) == 1 and hpsi.stride(0) == 1 and (nb <= 1 or hpsi.stride(1) == ld)
    _check(_apply(cell, _dptr(psi), ld, nb, _dptr(hpsi), _stream(stream)), "pw_apply_H")


_apply_na = _sig("pw_apply_H_noalloc", ct.c_int, [_vp, _vp, ct.c_int, ct.c_int, _vp, _vp])
_density = _sig("pw_density", ct.c_int, [_vp, _vp, ct.c_int, ct.c_int, _vp, _vp, _vp])


def pw_density(cell, psi, occ=None, rho=None, stream=None):
    """rho(r) = sum_b occ_b |psi_b(r)|^2 on the cell's grid; psi: CUDA complex128
    (npw, nb) column-major; occ: CUDA float64 (nb,) or None; returns rho as a
    CUDA float64 tensor of shape (N2, N1, N0) (x fastest)."""
    import torch
    npw, nb = psi.shape
    ld = psi.stride(1) if nb > 1 else npw
    assert psi.stride(0) == 1 and psi.is_cuda
    grid = pw_cell_info(cell)[1]
    if rho is None:
        rho = torch.empty((grid[2], grid[1], grid[0]), dtype=torch.float64, device=psi.device)
    optr = _dptr(occ) if occ is not None else ct.c_void_p()
    _check(_density(cell, _dptr(psi), ld, nb, optr, _dptr(rho), _stream(stream)), "pw_density")
    return rho


def pw_apply_H_noalloc(cell, psi, hpsi, stream=None):
    """hpsi <- H psi (FP64) using only the library's static scratch (no allocation)."""
    npw, nb = psi.shape
    ld = psi.stride(1) if nb > 1 else npw
    _check(_apply_na(cell, _dptr(psi), ld, nb, _dptr(hpsi), _stream(stream)), "pw_apply_H_noalloc")


def pw_destroy_cell(cell):
    _destroy(cell)


def _opts(nbands, tol, maxit, seed, x0, precision, chunk_rows=0, h_blocks=0):
    o = pw_solve_opts()
    o.nbands, o.tol, o.maxit, o.seed = int(nbands), float(tol), int(maxit), int(seed)
    o.precision = _PREC[precision]
    o.chunk_rows = int(chunk_rows)
    o.h_blocks = int(h_blocks)
    keep = None
    if x0 is not None and hasattr(x0, "data_ptr"):
        # a CUDA tensor (column-major, ld = npw): passed as a device pointer
        assert x0.stride(0) == 1 and (x0.shape[1] <= 1 or x0.stride(1) == x0.shape[0])
        keep = x0
        o.x0 = x0.data_ptr()
    elif x0 is not None:
        keep = np.asfortranarray(x0, dtype=np.complex128)
        o.x0 = keep.ctypes.data
    return o, keep


def pw_solver_create(cell, nbands, tol=1e-8, maxit=200, seed=0, x0=None, precision="fp64",
                     stream=None, chunk_rows=0, h_blocks=0):
    o, keep = _opts(nbands, tol, maxit, seed, x0, precision, chunk_rows, h_blocks)
    h = ct.c_void_p()
    _check(_screate(cell, ct.byref(o), _stream(stream), ct.byref(h)), "pw_solver_create")
    del keep
    return h


def pw_subspace_step(cell, solver):
    r = pw_step_report()
    _check(_sstep(cell, solver, ct.byref(r)), "pw_subspace_step")
    return r


_spolish = _sig("pw_solver_polish", ct.c_int, [_vp])


def pw_solver_polish(solver):
    _check(_spolish(solver), "pw_solver_polish")


def pw_solver_eigs(solver, nbands):
    e = np.zeros(nbands)
    r = np.zeros(nbands)
    _check(_seigs(solver, e.ctypes.data_as(ct.POINTER(ct.c_double)),
                  r.ctypes.data_as(ct.POINTER(ct.c_double))), "pw_solver_eigs")
    return e, r


def pw_solver_block(solver, out):
    _check(_sblock(solver, _dptr(out), out.shape[0]), "pw_solver_block")


_sset_p = _sig("pw_solver_set_p", ct.c_int, [_vp, _vp, ct.c_int])
_sget_p = _sig("pw_solver_get_p", ct.c_int, [_vp, _vp, ct.c_int, ct.POINTER(ct.c_int)])


def pw_solver_set_p(solver, p):
    """Replace the search directions P by p (CUDA complex128 (npw, nb), column-major,
    or a host numpy array)."""
    if isinstance(p, np.ndarray):
        keep = np.asfortranarray(p, dtype=np.complex128)
        _check(_sset_p(solver, ct.c_void_p(keep.ctypes.data), keep.shape[0]), "pw_solver_set_p")
        return
    assert p.stride(0) == 1
    _check(_sset_p(solver, _dptr(p), p.stride(1) if p.shape[1] > 1 else p.shape[0]), "pw_solver_set_p")


def pw_solver_get_p(solver, out):
    """Copy P into out (CUDA complex128 (npw, nb), column-major); returns whether P is defined."""
    have = ct.c_int()
    _check(_sget_p(solver, _dptr(out), out.shape[0], ct.byref(have)), "pw_solver_get_p")
    return bool(have.value)


def pw_solver_destroy(solver):
    _sdestroy(solver)


def pw_eigsolve(cell, nbands, tol=1e-8, maxit=200, seed=0, x0=None, precision="fp64",
                psi_out=None, stream=None, raise_noconv=True, chunk_rows=0, h_blocks=0):
    o, keep = _opts(nbands, tol, maxit, seed, x0, precision, chunk_rows, h_blocks)
    eig = np.zeros(nbands)
    rep = pw_solve_report()
    ptr = _dptr(psi_out) if psi_out is not None else ct.c_void_p()
    ld = psi_out.shape[0] if psi_out is not None else 0
    st = _eigsolve(cell, ct.byref(o), eig.ctypes.data_as(ct.POINTER(ct.c_double)), ptr, ld,
                   ct.byref(rep), _stream(stream))
    del keep
    if st != PW_OK and (st != PW_ERR_NOCONV or raise_noconv):
        raise PwError(st, "pw_eigsolve")
    return eig, rep, st


class Cell:
    """Owning wrapper around a pw_cell handle."""

    def __init__(self, L, tau, depth, dkb, ecut, vwidth=1.2, pwidth=1.2, grid=None,
                 precision="fp64", stream=None):
        self.h = pw_setup_cell(L, tau, depth, dkb, ecut, vwidth, pwidth, grid, precision, stream)
        self.npw, self.grid, self.m = pw_cell_info(self.h)
        self.nproj, _ = pw_cell_sizes(self.h)

    def apply_H(self, psi, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(psi)
        pw_apply_H(self.h, psi, out, stream)
        return out

    def set_precision(self, p):
        pw_cell_set_precision(self.h, p)

    def close(self):
        if self.h:
            pw_destroy_cell(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_hxc = _sig("pw_hxc_potential", ct.c_int, [_vp, _vp, _vp, _vp])
_set_hxc = _sig("pw_cell_set_hxc", ct.c_int, [_vp, _vp, _vp])


class pw_scf_opts(ct.Structure):
    _fields_ = [("nbands", ct.c_int), ("nocc", ct.c_int), ("fill", ct.c_double), ("mix", ct.c_double),
                ("maxiter", ct.c_int), ("tol", ct.c_double), ("eig_tol", ct.c_double),
                ("eig_maxit", ct.c_int), ("seed", ct.c_uint64), ("precision", ct.c_int)]


class pw_scf_report(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("eig_iters", ct.c_int), ("max_dn", ct.c_double)]


_scf = _sig("pw_scf", ct.c_int, [_vp, ct.POINTER(pw_scf_opts), ct.POINTER(ct.c_double), _vp,
                                  ct.POINTER(pw_scf_report), _vp])


def _grid_tensor(cell, device="cuda"):
    import torch
    g = pw_cell_info(cell)[1]
    return torch.empty((g[2], g[1], g[0]), dtype=torch.float64, device=device)


def pw_hxc_potential(cell, n, v=None, stream=None):
    """Model V_H + v_x of a density n (CUDA float64 grid tensor, (N2, N1, N0))."""
    if v is None:
        v = _grid_tensor(cell, n.device)
    _check(_hxc(cell, _dptr(n), _dptr(v), _stream(stream)), "pw_hxc_potential")
    return v


def pw_cell_set_hxc(cell, v=None, stream=None):
    """Local potential becomes V_loc + v (None restores V_loc)."""
    _check(_set_hxc(cell, _dptr(v) if v is not None else ct.c_void_p(), _stream(stream)), "pw_cell_set_hxc")


def pw_scf(cell, nbands, nocc, fill=2.0, mix=0.5, maxiter=30, tol=1e-6, eig_tol=1e-10, eig_maxit=200,
           seed=0, precision="fp64", stream=None, raise_noconv=True):
    """Linear-mixing SCF with the model V_Hxc; returns (eig (numpy), n_out (CUDA grid
    tensor), report, status)."""
    o = pw_scf_opts()
    o.nbands, o.nocc, o.fill, o.mix = int(nbands), int(nocc), float(fill), float(mix)
    o.maxiter, o.tol, o.eig_tol, o.eig_maxit = int(maxiter), float(tol), float(eig_tol), int(eig_maxit)
    o.seed, o.precision = int(seed), _PREC[precision]
    eig = np.zeros(nbands)
    n_out = _grid_tensor(cell)
    rep = pw_scf_report()
    st = _scf(cell, ct.byref(o), eig.ctypes.data_as(ct.POINTER(ct.c_double)), _dptr(n_out), ct.byref(rep),
              _stream(stream))
    if st != PW_OK and (st != PW_ERR_NOCONV or raise_noconv):
        raise PwError(st, "pw_scf")
    return eig, n_out, rep, st


_setproj = _sig("pw_cell_set_projectors", ct.c_int, [_vp, ct.c_int, _vp])


def pw_cell_set_projectors(cell, onthefly, stream=None):
    """Projectors resident (False) or regenerated in atom chunks per H psi (True)."""
    _check(_setproj(cell, 1 if onthefly else 0, _stream(stream)), "pw_cell_set_projectors")


# ---------------------------------------------------------------- autotuner --
class pw_fft_plan(ct.Structure):
    _fields_ = [("L", ct.c_int), ("R", ct.c_int), ("compact", ct.c_int), ("batch_bytes", ct.c_size_t)]


class pw_fft_tune_report(ct.Structure):
    _fields_ = [("ncand", ct.c_int), ("best", pw_fft_plan), ("dflt", pw_fft_plan),
                ("ms_best", ct.c_double), ("ms_default", ct.c_double)]


_fft_plans = _sig("pw_fft_plans", ct.c_int, [ct.c_int, ct.POINTER(pw_fft_plan), ct.c_int])
_set_fft_plan = _sig("pw_cell_set_fft_plan", ct.c_int, [_vp, ct.c_int, ct.POINTER(pw_fft_plan)])
_get_fft_plan = _sig("pw_cell_get_fft_plan", ct.c_int, [_vp, ct.c_int, ct.POINTER(pw_fft_plan)])
_tune_fft = _sig("pw_cell_autotune_fft", ct.c_int, [_vp, ct.c_int, ct.c_int, _vp,
                                                     ct.POINTER(pw_fft_tune_report)])
_tune_gemm = _sig("pw_autotune_gemm", ct.c_int, [ct.c_int, ct.c_int])
_tune_log = _sig("pw_cell_fft_tune_log", ct.c_int, [_vp, ct.c_char_p, ct.c_size_t])
_tune_table = _sig("pw_autotune_gemm_table", ct.c_int, [ct.c_char_p, ct.c_size_t])
_tune_load = _sig("pw_autotune_gemm_load", ct.c_int, [ct.c_char_p])


def pw_fft_plans(n):
    """Register line-FFT plans (L, R) compiled for grid size n."""
    k = _fft_plans(int(n), None, 0)
    arr = (pw_fft_plan * max(k, 1))()
    _fft_plans(int(n), arr, k)
    return [(arr[i].L, arr[i].R) for i in range(k)]


def pw_cell_set_fft_plan(cell, L, R, batch_bytes=0, precision="fp64", compact=False):
    """Set the cell's FFT plan (L = R = 0: Stockham passes; compact: sphere x-columns only)."""
    p = pw_fft_plan(int(L), int(R), 1 if compact else 0, int(batch_bytes))
    _check(_set_fft_plan(cell, _PREC[precision], ct.byref(p)), "pw_cell_set_fft_plan")


def pw_cell_get_fft_plan(cell, precision="fp64"):
    p = pw_fft_plan()
    _check(_get_fft_plan(cell, _PREC[precision], ct.byref(p)), "pw_cell_get_fft_plan")
    return (p.L, p.R, p.batch_bytes, bool(p.compact))


def pw_cell_autotune_fft(cell, nb, precision="fp64", stream=None):
    r = pw_fft_tune_report()
    _check(_tune_fft(cell, int(nb), _PREC[precision], _stream(stream), ct.byref(r)), "pw_cell_autotune_fft")
    return r


def pw_autotune_gemm(mode, split=1):
    """K split of the tensor-core GEMMs: 0 fixed (s = 1), 1 tuned per shape, 2 forced `split`."""
    _check(_tune_gemm(int(mode), int(split)), "pw_autotune_gemm")


def pw_autotune_gemm_table():
    n = _tune_table(None, 0)
    buf = ct.create_string_buffer(256 * (n + 1) + 1)
    _tune_table(buf, len(buf))
    return buf.value.decode()


def pw_cell_fft_tune_log(cell):
    """Candidates and times of the cell's last FFT tuning (text, one line each)."""
    n = _tune_log(cell, None, 0)
    buf = ct.create_string_buffer(n + 1)
    _tune_log(cell, buf, len(buf))
    return buf.value.decode()


_selftest_wait = _sig("pw_selftest_bounded_wait", ct.c_int, [ct.c_longlong, _vp])


def pw_selftest_bounded_wait(cycles, stream=None):
    """Status of the bounded-wait self-test (PW_ERR_TIMEOUT is the expected result)."""
    return int(_selftest_wait(int(cycles), _stream(stream)))


def pw_autotune_gemm_load(text):
    """Add K-split choices saved from pw_autotune_gemm_table; returns the lines added."""
    n = _tune_load(text.encode())
    if n < 0:
        raise PwError(PW_ERR_ARG, "pw_autotune_gemm_load")
    return n
