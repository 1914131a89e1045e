"""ctypes binding of libcute_gb.so (include/cute.h): argument marshalling only.

Every step of the pair-counting path runs in the CUDA library; this module
converts numpy arrays / torch tensors to pointers and statuses to
exceptions.  There is no fallback: if the library is missing or cannot be
built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcute_gb.so")

KINDS = {"mono": 0, "rmu": 1, "sigpi": 2, "theta": 3}
ESTIMATORS = {"periodic": 0, "natural": 1, "ls": 2}
STATUS = {0: "OK", -1: "INVALID", -2: "OOM", -3: "CUDA", -4: "STATE", -5: "TIMEOUT",
          -6: "UNSUPPORTED", -7: "DEVICE"}

# every exported symbol of include/cute.h
SYMBOLS = ["cute_ctx_create", "cute_ctx_destroy", "cute_last_error", "cute_sync",
           "cute_catalog_upload", "cute_catalog_free", "cute_catalog_size", "cute_grid_build",
           "cute_count_pairs", "cute_count_pairs_batched", "cute_count_pairs_adjoint",
           "cute_count_pairs_noalloc",
           "cute_last_stats", "cute_set_timing", "cute_set_launch", "cute_autotune",
           "cute_estimator", "cute_multipoles", "cute_sky_to_xyz", "cute_pixel_map",
           "cute_pixel_centres", "cute_estimator_weighted", "cute_density_grid_xi",
           "cute_theta_to_chord", "cute_version"]


class CuteError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("cute %s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


class PairDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("cat_a", ctypes.c_int32), ("cat_b", ctypes.c_int32),
                ("edges0", ctypes.c_void_p), ("n0", ctypes.c_int32),
                ("edges1", ctypes.c_void_p), ("n1", ctypes.c_int32),
                ("weighted", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("cells_per_reach", ctypes.c_int32), ("home_per_lane", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("slice", ctypes.c_int32),
                ("ms", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Cosmology(ctypes.Structure):
    _fields_ = [("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double),
                ("w0", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("candidate_pairs", ctypes.c_uint64), ("rechecked_pairs", ctypes.c_uint64),
                ("fp64_pairs", ctypes.c_uint64),
                ("pair_slots", ctypes.c_uint64), ("work_items", ctypes.c_uint64), ("launches", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("blocks", ctypes.c_int32),
                ("home_per_lane", ctypes.c_int32), ("kernel_ms", ctypes.c_float),
                ("stencil_pairs", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def lib():
    """Load libcute_gb.so (building it with nvcc if absent)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                from . import build as _b
                _b.build()
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            L.cute_ctx_create.argtypes = [ctypes.c_int, P, ctypes.POINTER(P)]
            L.cute_ctx_destroy.argtypes = [P]
            L.cute_last_error.argtypes = [P]
            L.cute_last_error.restype = ctypes.c_char_p
            L.cute_sync.argtypes = [P]
            L.cute_catalog_upload.argtypes = [P, P, P, i64, ctypes.c_int, f64,
                                              ctypes.POINTER(i32)]
            L.cute_catalog_free.argtypes = [P, i32]
            L.cute_catalog_size.argtypes = [P, i32, ctypes.POINTER(i64)]
            L.cute_grid_build.argtypes = [P, P, i32, P, i32]
            L.cute_count_pairs.argtypes = [P, ctypes.POINTER(PairDesc), P, P, P]
            L.cute_count_pairs_batched.argtypes = [P, i32, P, P, P]
            L.cute_count_pairs_adjoint.argtypes = [P, ctypes.POINTER(PairDesc), P, P, P]
            L.cute_count_pairs_noalloc.argtypes = [P, ctypes.POINTER(PairDesc), P, P]
            L.cute_last_stats.argtypes = [P, ctypes.POINTER(Stats)]
            L.cute_set_timing.argtypes = [P, i32]
            L.cute_set_launch.argtypes = [P, i32, i32, i32, i32]
            L.cute_autotune.argtypes = [P, i32, P, i32, i64, ctypes.POINTER(Tuning)]
            L.cute_estimator.argtypes = [ctypes.c_int, P, P, P, i64, i64, i32, P, f64, P]
            L.cute_theta_to_chord.argtypes = [P, i32, P]
            L.cute_multipoles.argtypes = [P, i32, i32, P, i32, P, P]
            L.cute_sky_to_xyz.argtypes = [P, P, P, P, i64, P, P]
            L.cute_pixel_map.argtypes = [P, P, P, i64, i32, P]
            L.cute_pixel_centres.argtypes = [P, i32, P, i64, P]
            L.cute_density_grid_xi.argtypes = [P, P, P, i64, f64, i32, P, i32, P, P]
            L.cute_estimator_weighted.argtypes = [ctypes.c_int, P, P, P, f64, f64, f64, f64,
                                                  i32, P]
            L.cute_version.restype = ctypes.c_char_p
            for name in SYMBOLS:
                if name not in ("cute_last_error", "cute_version"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(st, ctx=None):
    if st != 0:
        msg = lib().cute_last_error(ctx).decode(errors="replace") if ctx is not None else ""
        raise CuteError(st, msg)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Data pointer of a numpy array or torch tensor (kept alive by caller)."""
    if x is None:
        return None
    if _is_torch(x):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


def _xyz(x):
    if _is_torch(x):
        import torch
        x = x.detach()
        if x.dtype != torch.float64:
            x = x.to(torch.float64)
        x = x.contiguous()
        if x.ndim != 2 or x.shape[1] != 3:
            raise ValueError("positions must be (n, 3)")
        return x
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 2 or x.shape[1] != 3:
        raise ValueError("positions must be (n, 3)")
    return x


def _w(w):
    if w is None:
        return None
    if _is_torch(w):
        import torch
        return w.detach().to(torch.float32).contiguous()
    return np.ascontiguousarray(w, dtype=np.float32)


class Catalog:
    def __init__(self, ctx, cid, n, periodic, L):
        self.ctx, self.id, self.n, self.periodic, self.L = ctx, cid, n, periodic, L

    def free(self):
        if self.id is not None and self.ctx.handle:
            _check(lib().cute_catalog_free(self.ctx.handle, self.id), self.ctx.handle)
        self.id = None


class Context:
    """A counting context on one CUDA device (owns catalogs and buffers).

    stream: None -> the torch current stream of the device when torch is
    available (so library work is ordered with torch work), else a stream the
    library creates; or an integer cudaStream_t handle."""

    # cudaStreamLegacy: the handle of the legacy default stream, whose
    # cudaStream_t value 0 the C ABI reads as "create a stream"
    _LEGACY_STREAM = 0x1

    def __init__(self, device: int = 0, stream=None):
        L = lib()
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
                    if stream == 0:
                        stream = self._LEGACY_STREAM
            except Exception:
                stream = None
        h = ctypes.c_void_p()
        st = L.cute_ctx_create(int(device), ctypes.c_void_p(stream) if stream else None,
                               ctypes.byref(h))
        if st != 0:
            raise CuteError(st, L.cute_last_error(None).decode(errors="replace"))
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            lib().cute_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -------------------------------------------------------------- catalogs
    def upload(self, xyz, weights=None, periodic=False, L=0.0) -> Catalog:
        x = _xyz(xyz)
        w = _w(weights)
        cid = ctypes.c_int32()
        _check(lib().cute_catalog_upload(self.handle, _ptr(x), _ptr(w), int(x.shape[0]),
                                         0 if periodic else 1, float(L), ctypes.byref(cid)),
               self.handle)
        return Catalog(self, cid.value, int(x.shape[0]), periodic, L)

    def grid(self, cats, reach, cells_per_reach: int = 0):
        ids = (ctypes.c_int32 * len(cats))(*[c.id for c in cats])
        r = np.ascontiguousarray(np.broadcast_to(np.asarray(reach, dtype=np.float64), (3,)))
        _check(lib().cute_grid_build(self.handle, ids, len(cats), _ptr(r), int(cells_per_reach)),
               self.handle)

    # -------------------------------------------------------------- counting
    @staticmethod
    def _desc(kind, a, b, e0, e1, weighted):
        d = PairDesc()
        d.kind = KINDS[kind]
        d.cat_a = a.id
        d.cat_b = (b if b is not None else a).id
        d.edges0 = e0.ctypes.data
        d.n0 = len(e0) - 1
        if e1 is not None:
            d.edges1 = e1.ctypes.data
            d.n1 = len(e1) - 1
        else:
            d.edges1 = None
            d.n1 = 0
        d.weighted = int(weighted)
        return d

    def count(self, kind, a, b=None, edges0=None, edges1=None, weighted=False, out=None,
              wsum_out=None, want_oor=True):
        """Pair counts of a x b (b None: auto).  Returns (counts, oor, wsum).
        counts has shape (n0, n1) (n1 = 1 for 1-D kinds).  out / wsum_out may
        be preallocated numpy arrays or CUDA torch tensors (uint64 / float64,
        viewed as int64 for torch)."""
        e0 = np.ascontiguousarray(edges0, dtype=np.float64)
        e1 = None if edges1 is None else np.ascontiguousarray(edges1, dtype=np.float64)
        n0 = len(e0) - 1
        n1 = (len(e1) - 1) if (e1 is not None and kind in ("rmu", "sigpi")) else 1
        d = self._desc(kind, a, b, e0, e1 if kind in ("rmu", "sigpi") else None, weighted)
        counts = out if out is not None else np.zeros(n0 * n1, dtype=np.uint64)
        wsum = None
        if weighted:
            wsum = wsum_out if wsum_out is not None else np.zeros(n0 * n1, dtype=np.float64)
        oor = ctypes.c_uint64(0)
        _check(lib().cute_count_pairs(self.handle, ctypes.byref(d), _ptr(counts),
                                      ctypes.byref(oor) if want_oor else None, _ptr(wsum)),
               self.handle)
        if not _is_torch(counts):
            counts = counts.reshape(n0, n1)
            if wsum is not None and not _is_torch(wsum):
                wsum = wsum.reshape(n0, n1)
        return counts, (int(oor.value) if want_oor else None), wsum

    def count_batched(self, kind, pairs, edges0, edges1=None, weighted=False, device=False):
        """pairs: list of (a, b) catalogs (b None: auto), counted in one launch.
        Returns a list of (n0, n1) uint64 arrays (and wsum arrays if weighted).
        device=True: outputs are CUDA tensors (int64 viewing uint64 counts);
        repeated identical calls then replay a captured CUDA graph."""
        e0 = np.ascontiguousarray(edges0, dtype=np.float64)
        e1 = None if edges1 is None else np.ascontiguousarray(edges1, dtype=np.float64)
        n0 = len(e0) - 1
        n1 = (len(e1) - 1) if (e1 is not None and kind in ("rmu", "sigpi")) else 1
        n = len(pairs)
        descs = (PairDesc * n)()
        for i, (a, b) in enumerate(pairs):
            descs[i] = self._desc(kind, a, b, e0, e1 if kind in ("rmu", "sigpi") else None,
                                  weighted)
        if device:
            import torch
            if not hasattr(self, "_dev_outs") or self._dev_outs[0] != (n, n0 * n1, weighted):
                outs = [torch.zeros(n0 * n1, dtype=torch.int64, device="cuda") for _ in range(n)]
                wso = ([torch.zeros(n0 * n1, dtype=torch.float64, device="cuda") for _ in range(n)]
                       if weighted else None)
                self._dev_outs = ((n, n0 * n1, weighted), outs, wso)
            _, outs, ws = self._dev_outs
            optr = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
            wptr = (ctypes.c_void_p * n)(*[o.data_ptr() for o in ws]) if weighted else None
            _check(lib().cute_count_pairs_batched(self.handle, n, descs, optr, wptr), self.handle)
            res = [o.view(n0, n1) for o in outs]
            return (res, [w.view(n0, n1) for w in ws]) if weighted else res
        outs = [np.zeros(n0 * n1, dtype=np.uint64) for _ in range(n)]
        optr = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
        ws, wptr = None, None
        if weighted:
            ws = [np.zeros(n0 * n1, dtype=np.float64) for _ in range(n)]
            wptr = (ctypes.c_void_p * n)(*[o.ctypes.data for o in ws])
        _check(lib().cute_count_pairs_batched(self.handle, n, descs, optr, wptr), self.handle)
        res = [o.reshape(n0, n1) for o in outs]
        if weighted:
            return res, [w.reshape(n0, n1) for w in ws]
        return res

    def adjoint(self, kind, a, b=None, edges0=None, edges1=None, G=None, grad_b=False):
        """Gradient of sum_b G_b W_b with respect to the weights of a (and of b
        for cross counts when grad_b)."""
        e0 = np.ascontiguousarray(edges0, dtype=np.float64)
        e1 = None if edges1 is None else np.ascontiguousarray(edges1, dtype=np.float64)
        d = self._desc(kind, a, b, e0, e1 if kind in ("rmu", "sigpi") else None, True)
        if _is_torch(G):
            import torch
            Gc = G.detach().to(torch.float64).contiguous()
            ga = torch.zeros(a.n, dtype=torch.float64, device=G.device)
            gb = (torch.zeros(b.n, dtype=torch.float64, device=G.device)
                  if (grad_b and b is not None) else None)
        else:
            Gc = np.ascontiguousarray(G, dtype=np.float64).ravel()
            ga = np.zeros(a.n, dtype=np.float64)
            gb = np.zeros(b.n, dtype=np.float64) if (grad_b and b is not None) else None
        _check(lib().cute_count_pairs_adjoint(self.handle, ctypes.byref(d), _ptr(Gc), _ptr(ga),
                                              _ptr(gb)), self.handle)
        return (ga, gb) if grad_b else ga

    def autotune(self, kind, pairs, edges0, edges1=None, weighted=False, tune_cells=True,
                 max_items=20000):
        """Time launch shapes (and 2, 3, 4 cells per reach if tune_cells) on
        these pair sets and keep the fastest for later counts."""
        e0 = np.ascontiguousarray(edges0, dtype=np.float64)
        e1 = None if edges1 is None else np.ascontiguousarray(edges1, dtype=np.float64)
        descs = (PairDesc * len(pairs))()
        for i, (a, b) in enumerate(pairs):
            descs[i] = self._desc(kind, a, b, e0, e1 if kind in ("rmu", "sigpi") else None,
                                  weighted)
        t = Tuning()
        _check(lib().cute_autotune(self.handle, len(pairs), descs, int(bool(tune_cells)),
                                   int(max_items), ctypes.byref(t)), self.handle)
        return t.as_dict()

    # -------------------------------------------------------------- sky input
    def sky_to_xyz(self, ra, dec, z=None, omega_m=0.3, omega_l=0.7, w0=-1.0):
        """(RA, Dec) in degrees and redshifts z (None: unit vectors) -> (n, 3)
        float64 comoving positions in Mpc/h, on the GPU.  numpy in, numpy
        out; CUDA tensors in, CUDA tensor out."""
        cos = Cosmology(omega_m, omega_l, w0)
        if _is_torch(ra):
            import torch
            conv = lambda a: a.detach().to(torch.float64).contiguous()
            r, d = conv(ra), conv(dec)
            zz = conv(z) if z is not None else None
            out = torch.empty((r.shape[0], 3), dtype=torch.float64, device=r.device)
        else:
            r = np.ascontiguousarray(ra, dtype=np.float64)
            d = np.ascontiguousarray(dec, dtype=np.float64)
            zz = None if z is None else np.ascontiguousarray(z, dtype=np.float64)
            out = np.empty((len(r), 3), dtype=np.float64)
        if len(d) != len(r) or (zz is not None and len(zz) != len(r)):
            raise ValueError("ra, dec and z must have the same length")
        _check(lib().cute_sky_to_xyz(self.handle, _ptr(r), _ptr(d), _ptr(zz), len(r),
                                     ctypes.byref(cos), _ptr(out)), self.handle)
        return out

    # -------------------------------------------------------------- pixel maps
    def pixel_map(self, xyz, weights=None, nside=256):
        """HEALPix RING map (12 nside^2 doubles) of unit vectors, each pixel
        the summed weight of its objects.  numpy in -> numpy out, CUDA
        tensors in -> CUDA tensor out."""
        x = _xyz(xyz)
        w = _w(weights)
        npix = 12 * nside * nside
        if _is_torch(x):
            import torch
            out = torch.zeros(npix, dtype=torch.float64, device=x.device)
        else:
            out = np.zeros(npix, dtype=np.float64)
        _check(lib().cute_pixel_map(self.handle, _ptr(x), _ptr(w), int(x.shape[0]), int(nside),
                                    _ptr(out)), self.handle)
        return out

    def pixel_centres(self, nside, pix):
        """Unit-vector centres (m, 3) of HEALPix RING pixels."""
        if _is_torch(pix):
            import torch
            p = pix.detach().to(torch.int64).contiguous()
            out = torch.empty((p.shape[0], 3), dtype=torch.float64, device=p.device)
        else:
            p = np.ascontiguousarray(pix, dtype=np.int64)
            out = np.empty((len(p), 3), dtype=np.float64)
        _check(lib().cute_pixel_centres(self.handle, int(nside), _ptr(p), len(p), _ptr(out)),
               self.handle)
        return out

    # -------------------------------------------------------------- density grid
    def density_grid_xi(self, xyz, L, ngrid, edges, weights=None):
        """xi(r) of a periodic box from a TSC density grid (Sec. 3.4.4).
        Returns (xi, lag vectors per bin)."""
        x = _xyz(xyz)
        w = _w(weights)
        e = np.ascontiguousarray(edges, dtype=np.float64)
        xi = np.zeros(len(e) - 1)
        lags = np.zeros(len(e) - 1)
        _check(lib().cute_density_grid_xi(self.handle, _ptr(x), _ptr(w), int(x.shape[0]), float(L),
                                          int(ngrid), _ptr(e), len(e) - 1, _ptr(xi), _ptr(lags)),
               self.handle)
        return xi, lags

    # -------------------------------------------------------------- misc
    def sync(self):
        _check(lib().cute_sync(self.handle), self.handle)

    def stats(self) -> dict:
        s = Stats()
        _check(lib().cute_last_stats(self.handle, ctypes.byref(s)), self.handle)
        return s.as_dict()

    def set_timing(self, on: bool):
        _check(lib().cute_set_timing(self.handle, int(bool(on))), self.handle)

    def set_launch(self, home_per_lane=0, warps_per_block=0, slice=0, table_binning=False):
        _check(lib().cute_set_launch(self.handle, int(home_per_lane), int(warps_per_block),
                                     int(slice), int(bool(table_binning))), self.handle)
        self.table_binning = bool(table_binning)


def estimator(kind, DD, DR=None, RR=None, Nd=0, Nr=0, edges=None, L=0.0):
    """Eq. 13 ('periodic'), Eq. 14 ('natural') or Eq. 15 ('ls') from counts."""
    DD = np.ascontiguousarray(DD, dtype=np.uint64).ravel()
    DR_ = None if DR is None else np.ascontiguousarray(DR, dtype=np.uint64).ravel()
    RR_ = None if RR is None else np.ascontiguousarray(RR, dtype=np.uint64).ravel()
    e = None if edges is None else np.ascontiguousarray(edges, dtype=np.float64)
    out = np.zeros(len(DD), dtype=np.float64)
    _check(lib().cute_estimator(ESTIMATORS[kind], _ptr(DD), _ptr(DR_), _ptr(RR_), int(Nd),
                                int(Nr), len(DD), _ptr(e), float(L), _ptr(out)))
    return out


def multipoles(xi, mu_edges, ells=(0, 2, 4)):
    """Even multipoles xi_l(r) of a binned xi(r, mu) (Eq. 3), xi of shape
    (n_r, n_mu) on mu edges from 0 to 1.  Returns (len(ells), n_r)."""
    x = np.ascontiguousarray(xi, dtype=np.float64)
    if x.ndim != 2:
        raise ValueError("xi must be (n_r, n_mu)")
    m = np.ascontiguousarray(mu_edges, dtype=np.float64)
    if len(m) != x.shape[1] + 1:
        raise ValueError("mu_edges must have n_mu + 1 values")
    ls = np.ascontiguousarray(ells, dtype=np.int32)
    out = np.zeros((len(ls), x.shape[0]), dtype=np.float64)
    _check(lib().cute_multipoles(_ptr(x), x.shape[0], x.shape[1], _ptr(m), len(ls), _ptr(ls),
                                 _ptr(out)))
    return out


def estimator_weighted(kind, DD, DR, RR, s_d, q_d, s_r, q_r):
    """Eq. 14 ('natural') or Eq. 15 ('ls') on weighted pair sums, each
    normalised by its total pair weight (S: sum of weights, Q: of squares)."""
    DD = np.ascontiguousarray(DD, dtype=np.float64).ravel()
    DR_ = None if DR is None else np.ascontiguousarray(DR, dtype=np.float64).ravel()
    RR = np.ascontiguousarray(RR, dtype=np.float64).ravel()
    out = np.zeros(len(DD), dtype=np.float64)
    _check(lib().cute_estimator_weighted(ESTIMATORS[kind], _ptr(DD), _ptr(DR_), _ptr(RR),
                                         float(s_d), float(q_d), float(s_r), float(q_r), len(DD),
                                         _ptr(out)))
    return out


def theta_to_chord(theta_deg):
    t = np.ascontiguousarray(theta_deg, dtype=np.float64)
    out = np.zeros(len(t), dtype=np.float64)
    _check(lib().cute_theta_to_chord(_ptr(t), len(t), _ptr(out)))
    return out


def version() -> str:
    return lib().cute_version().decode()


class _HeldCatalogs:
    """Catalogs a forward pass keeps for its backward.  They are freed when
    the backward has used them, or, if no backward ever runs, when the
    autograd graph that holds this object is released (weakref finaliser),
    so an undifferentiated forward leaves nothing on the device."""

    def __init__(self, *cats):
        self.cats = [c for c in cats if c is not None]
        self._fin = weakref.finalize(self, _HeldCatalogs._free, self.cats)

    @staticmethod
    def _free(cats):
        for c in cats:
            try:
                c.free()
            except Exception:  # the context may already be closed
                pass

    def release(self):
        self._fin()


def _make_weighted_count():
    import torch

    class CuteWeightedCount(torch.autograd.Function):
        """W_b = sum of w_i w_j over the pairs in bin b (auto: unique pairs of
        one catalog; cross: all pairs of two), differentiable in the weights.

        forward: upload + grid + cute_count_pairs (weighted), outputs on the
        weights' device; backward: cute_count_pairs_adjoint with the upstream
        gradient G = dL/dW, giving dL/dw_i = sum_j w_j G[bin(i, j)].

        apply(wa, wb, ctx, kind, xyz_a, xyz_b, edges0, edges1, periodic, L,
        reach, cells_per_reach): wb / xyz_b None for an auto count; edges1
        None for 1-D kinds; reach as for Context.grid.  Returns W as an
        (n0, n1) float64 tensor."""

        @staticmethod
        def forward(fctx, wa, wb, ctx, kind, xyz_a, xyz_b, edges0, edges1, periodic, L, reach,
                    cells_per_reach=0):
            A = ctx.upload(xyz_a, weights=wa, periodic=periodic, L=L)
            B = ctx.upload(xyz_b, weights=wb, periodic=periodic, L=L) if xyz_b is not None else None
            ctx.grid([A] if B is None else [A, B], reach, cells_per_reach)
            e0 = np.ascontiguousarray(edges0, dtype=np.float64)
            e1 = None if edges1 is None else np.ascontiguousarray(edges1, dtype=np.float64)
            n0 = len(e0) - 1
            n1 = (len(e1) - 1) if (e1 is not None and kind in ("rmu", "sigpi")) else 1
            cnt = torch.zeros(n0 * n1, dtype=torch.int64, device=wa.device)
            W = torch.zeros(n0 * n1, dtype=torch.float64, device=wa.device)
            ctx.count(kind, A, B, e0, e1, weighted=True, out=cnt, wsum_out=W, want_oor=False)
            if fctx.needs_input_grad[0] or fctx.needs_input_grad[1]:
                fctx.cute = (ctx, kind, A, B, e0, e1, wa.dtype, None if wb is None else wb.dtype)
                fctx.held = _HeldCatalogs(A, B)
            else:
                A.free()
                if B is not None:
                    B.free()
            return W.view(n0, n1)

        @staticmethod
        def backward(fctx, gW):
            ctx, kind, A, B, e0, e1, da, db = fctx.cute
            G = gW.detach().to(torch.float64).contiguous().view(-1)
            if B is None:
                ga, gb = ctx.adjoint(kind, A, None, e0, e1, G=G), None
            else:
                ga, gb = ctx.adjoint(kind, A, B, e0, e1, G=G, grad_b=True)
            fctx.held.release()
            fctx.cute = None
            return (ga.to(da), None if gb is None else gb.to(db)) + (None,) * 10

    return CuteWeightedCount


def __getattr__(name):
    # torch is imported only when the autograd wrapper is asked for
    if name == "CuteWeightedCount":
        cls = _make_weighted_count()
        globals()[name] = cls
        return cls
    raise AttributeError(name)
