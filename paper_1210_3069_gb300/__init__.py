"""Python binding of libcalclens_gb300.so (GB300 lens-plane library).

Argument marshalling only: torch supplies device memory and the stream, and
every step of the computation runs in the library's CUDA kernels.  Importing
works without a GPU; calls need the built library (``build()``) and a CUDA
device, and raise ``CalclensError`` otherwise - there is no CPU fallback.

Names follow the C ABI in include/calclens.h (``clc_<name>`` -> ``<name>``).
"""
import ctypes
import os

import torch

from . import builder as _build

LIB_PATH = _build.LIB
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, ETIMEOUT = range(6)
RING, NEST = 0, 1
FP64, FP32, MIXED = 0, 1, 2
PLAN_GRAPH, PLAN_TUNE = 1, 2
SOLVER_SHT, SOLVER_SHTMG = 0, 1
STOP_RESIDUAL, STOP_TAU = 0, 1

_p = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_d = ctypes.c_double


class CalclensError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"calclens status {code}: {msg}")
        self.code = code


class Derivs(ctypes.Structure):
    _fields_ = [("a_th", _p), ("a_ph", _p), ("u_tt", _p), ("u_pp", _p), ("u_tp", _p)]


class MGParams(ctypes.Structure):
    _fields_ = [("nside_sht", _i), ("lmax", _i), ("nside_bundle", _i), ("ncell", _i), ("nu1", _i), ("nu2", _i),
                ("max_cycles", _i), ("fixed_cycles", _i), ("tol", _d), ("precision", _i), ("stop_rule", _i),
                ("eps", _d), ("refine_cycles", _i)]


class Rays(ctypes.Structure):
    _fields_ = [("n", _i64), ("x", _p), ("beta", _p), ("A", _p), ("Ap", _p), ("bundle", _p)]


_SIGS = {
    "clc_create": (_i, [ctypes.POINTER(_p), _i, _p]),
    "clc_destroy": (_i, [_p]),
    "clc_sync": (_i, [_p]),
    "clc_last_error": (ctypes.c_char_p, [_p]),
    "clc_release_caches": (_i, [_p]),
    "clc_bin_particles": (_i, [_p, _p, _p, _i64, _i, _i, _p]),
    "clc_counts_to_kappa": (_i, [_p, _p, _i, _d, _d, _p]),
    "clc_degrade": (_i, [_p, _p, _i, _p, _i]),
    "clc_smooth_particles": (_i, [_p, _p, _p, _i64, _i, _d, _p, _p]),
    "clc_density_to_kappa": (_i, [_p, _p, _i, _d, _d, _p]),
    "clc_find_images": (_i, [_p, _i, _p, _p, _i64, _p, _i, _p, _p, _p, _p]),
    "clc_set_table_budget": (_i, [_p, ctypes.c_size_t]),
    "clc_sht_analysis": (_i, [_p, _p, _i, _i, _p]),
    "clc_sht_synthesis": (_i, [_p, _p, _i, _i, _p]),
    "clc_poisson_sht": (_i, [_p, _p, _i, _i, _i, _p, ctypes.POINTER(Derivs)]),
    "clc_poisson_sht_batch": (_i, [_p, ctypes.POINTER(_p), _i, _i, _i, _i, ctypes.POINTER(_p),
                                   ctypes.POINTER(Derivs)]),
    "clc_solution_create": (_i, [_p, _i, ctypes.POINTER(MGParams), ctypes.POINTER(_p)]),
    "clc_solution_destroy": (_i, [_p]),
    "clc_solution_create_domain": (_i, [_p, _i, ctypes.POINTER(MGParams), ctypes.POINTER(ctypes.c_int32), _i,
                                        ctypes.POINTER(_p)]),
    "clc_solution_domain": (_i, [_p, ctypes.POINTER(_i), ctypes.POINTER(_i64)]),
    "clc_counts_to_kappa_masked": (_i, [_p, _p, _p, _i, _d, _p]),
    "clc_solution_info": (_i, [_p, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "clc_poisson_shtmg": (_i, [_p, _p, _i, ctypes.POINTER(MGParams), _p, ctypes.POINTER(Derivs)]),
    "clc_lens_derivs": (_i, [_p, _p, _p, _p, _p, _i64, ctypes.POINTER(Derivs)]),
    "clc_rays_init": (_i, [_p, _p, _p, _d, _i, ctypes.POINTER(Rays)]),
    "clc_rays_init_pixels": (_i, [_p, _i, _d, _i, ctypes.POINTER(Rays)]),
    "clc_ray_step": (_i, [_p, _p, ctypes.POINTER(Derivs), _i, _d, _d, _d, ctypes.POINTER(Rays)]),
    "clc_raytrace_planes": (_i, [_p, _i, ctypes.POINTER(MGParams), ctypes.POINTER(_p), _i, _i, ctypes.POINTER(_d),
                                 ctypes.POINTER(Rays)]),
    "clc_sht_plan_create": (_i, [_p, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), _i, _i, ctypes.POINTER(_p)]),
    "clc_sht_plan_execute": (_i, [_p, ctypes.POINTER(_p), ctypes.POINTER(_p), ctypes.POINTER(Derivs)]),
    "clc_sht_plan_info": (_i, [_p, ctypes.POINTER(_i), ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_size_t)]),
    "clc_sht_plan_destroy": (_i, [_p]),
    "clc_gal_trace": (_i, [_p, _i, ctypes.POINTER(_p), _i, _i, _i, ctypes.POINTER(_d), _i64, _p, _p, _p, _p,
                           ctypes.POINTER(_p)]),
    "clc_gal_trace_adjoint": (_i, [_p, _p, ctypes.POINTER(_p)]),
    "clc_gal_trace_mg": (_i, [_p, _i, ctypes.POINTER(_p), _i, ctypes.POINTER(MGParams), ctypes.POINTER(_d), _i64, _p,
                              _p, _p, _p, ctypes.POINTER(_p)]),
    "clc_gal_tape_destroy": (_i, [_p]),
    "clc_gemm_f16x3": (_i, [_p, _p, _p, _p, _p, _i, _i, _i, _i, _p]),
    "clc_eb_analysis": (_i, [_p, _p, _p, _i, _i, _p, _p]),
    "clc_power_spectrum": (_i, [_p, _p, _p, _i, _p]),
    "clc_lensing_spectra": (_i, [_p, _p, _p, _i, _i, _p]),
    "clc_profile": (_i, [_p, _i]),
    "clc_profile_query": (_i, [_p, ctypes.c_char_p, ctypes.POINTER(_i64), ctypes.POINTER(_d)]),
    "clc_launch_count": (_i64, [_p]),
    "clc_diag_bounded_wait": (_i, [_p, _i64]),
}


def exported_symbols():
    """Names of the C entry points the binding expects in the library."""
    return list(_SIGS)


def lib():
    """Load the shared library (it must have been built with ``build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise CalclensError(ECUDA, f"{LIB_PATH} is missing: run paper_1210_3069_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH, mode=ctypes.RTLD_GLOBAL)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def build(force=False):
    """Compile the CUDA library in-tree (see builder.py)."""
    global _lib
    path = _build.build(force=force)
    return path


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise CalclensError(EINVAL, "tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise CalclensError(EINVAL, "tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """A library context bound to a CUDA device and (by default) torch's
    current stream on it."""

    def __init__(self, device=0, stream=None):
        if not torch.cuda.is_available():
            raise CalclensError(ECUDA, "no CUDA device: the library has no CPU path")
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = ctypes.c_void_p()
        self._check(lib().clc_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream)), None)
        self.h = h

    def _check(self, rc, h=-1):
        if rc != OK:
            hh = self.h if h == -1 else h
            msg = lib().clc_last_error(hh).decode() if hh else ""
            raise CalclensError(rc, msg)
        return rc

    def close(self):
        if getattr(self, "h", None):
            lib().clc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        return self._check(lib().clc_sync(self.h))

    def release_caches(self):
        return self._check(lib().clc_release_caches(self.h))

    def profile(self, enable=True):
        return self._check(lib().clc_profile(self.h, 1 if enable else 0))

    def profile_query(self, name):
        """(launches, total device ms) recorded for kernel `name`."""
        n = _i64()
        ms = _d()
        self._check(lib().clc_profile_query(self.h, name.encode(), ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def launch_count(self):
        return int(lib().clc_launch_count(self.h))

    def diag_bounded_wait(self, polls):
        """Run the bounded mbarrier wait that nothing completes (the timeout
        path of the pipelined kernels); the next sync raises CLC_ETIMEOUT."""
        self._check(lib().clc_diag_bounded_wait(self.h, int(polls)))

    # -- step 1 -----------------------------------------------------------
    def bin_particles(self, z, phi, nside, ordering=RING, counts=None):
        if counts is None:
            counts = torch.zeros(12 * nside * nside, dtype=torch.int32, device=self.device)
        self._check(lib().clc_bin_particles(self.h, _ptr(z), _ptr(phi), z.numel(), nside, ordering, _ptr(counts)))
        return counts

    def counts_to_kappa(self, counts, nside, nbar, scale, kappa=None):
        if kappa is None:
            kappa = torch.empty(12 * nside * nside, dtype=torch.float64, device=self.device)
        self._check(lib().clc_counts_to_kappa(self.h, _ptr(counts), nside, float(nbar), float(scale), _ptr(kappa)))
        return kappa

    def counts_to_kappa_masked(self, counts, covered, nside, scale, kappa=None):
        """Partial-sky source: kappa from the counts of the covered pixels
        (covered: uint8/bool map), 0 elsewhere, with the covered region's own
        mean density."""
        if kappa is None:
            kappa = torch.empty(12 * nside * nside, dtype=torch.float64, device=self.device)
        cov = covered.to(torch.uint8).contiguous()
        self._check(lib().clc_counts_to_kappa_masked(self.h, _ptr(counts), _ptr(cov), nside, float(scale),
                                                     _ptr(kappa)))
        return kappa

    def smooth_particles(self, z, phi, nside, sigma=0.0, sigma_each=None, rho=None):
        """Epanechnikov-smoothed particle number per RING pixel (accumulated
        into rho, a new zero map if None)."""
        if rho is None:
            rho = torch.zeros(12 * nside * nside, dtype=torch.float64, device=self.device)
        self._check(lib().clc_smooth_particles(self.h, _ptr(z), _ptr(phi), z.numel(), int(nside), float(sigma),
                                               _ptr(sigma_each) if sigma_each is not None else None, _ptr(rho)))
        return rho

    def density_to_kappa(self, rho, nside, nbar, scale, kappa=None):
        if kappa is None:
            kappa = torch.empty(12 * nside * nside, dtype=torch.float64, device=self.device)
        self._check(lib().clc_density_to_kappa(self.h, _ptr(rho), int(nside), float(nbar), float(scale), _ptr(kappa)))
        return kappa

    def degrade(self, fine, nside_fine, nside_coarse, out=None):
        if out is None:
            out = torch.empty(12 * nside_coarse ** 2, dtype=torch.float64, device=self.device)
        self._check(lib().clc_degrade(self.h, _ptr(fine), nside_fine, _ptr(out), nside_coarse))
        return out

    # -- step 2 -----------------------------------------------------------
    def sht_analysis(self, m, nside, lmax):
        alm = torch.empty((lmax + 1) * (lmax + 2) // 2, dtype=torch.complex128, device=self.device)
        self._check(lib().clc_sht_analysis(self.h, _ptr(m), nside, lmax, _ptr(alm)))
        return alm

    def set_table_budget(self, nbytes):
        """Limit the FP64 Legendre table to nbytes (0: automatic); larger
        tables are processed one order range at a time."""
        self._check(lib().clc_set_table_budget(self.h, int(nbytes)))

    def sht_synthesis(self, alm, nside, lmax):
        out = torch.empty(12 * nside * nside, dtype=torch.float64, device=self.device)
        self._check(lib().clc_sht_synthesis(self.h, _ptr(alm), nside, lmax, _ptr(out)))
        return out

    def _derivs(self, n, want):
        t = {k: torch.empty(n, dtype=torch.float64, device=self.device) for k in want}
        d = Derivs(*[(_ptr(t[k]) if k in t else None) for k in ("a_th", "a_ph", "u_tt", "u_pp", "u_tp")])
        return t, d

    def poisson_sht(self, kappa, nside, lmax, precision=FP64, derivatives=True, psi=True):
        npx = 12 * nside * nside
        out, d = self._derivs(npx, ("a_th", "a_ph", "u_tt", "u_pp", "u_tp") if derivatives else ())
        p = torch.empty(npx, dtype=torch.float64, device=self.device) if psi else None
        self._check(lib().clc_poisson_sht(self.h, _ptr(kappa), nside, lmax, precision, _ptr(p),
                                          ctypes.byref(d) if derivatives else None))
        if psi:
            out["psi"] = p
        return out

    def poisson_sht_batch(self, kappa, nside, lmax, precision=MIXED, derivatives=True, psi=True):
        """clc_poisson_sht_batch over the rows of kappa[P, 12 nside^2]; returns
        a dict of [P, 12 nside^2] tensors (psi and/or the five lens fields)."""
        P, npx = kappa.shape
        names = ("a_th", "a_ph", "u_tt", "u_pp", "u_tp") if derivatives else ()
        out = {k: torch.empty(P, npx, dtype=torch.float64, device=self.device) for k in names}
        if psi:
            out["psi"] = torch.empty(P, npx, dtype=torch.float64, device=self.device)
        kp = (_p * P)(*[kappa[i].data_ptr() for i in range(P)])
        pp = (_p * P)(*[out["psi"][i].data_ptr() for i in range(P)]) if psi else None
        dd = (Derivs * P)(*[Derivs(*[out[k][i].data_ptr() for k in names]) for i in range(P)]) if derivatives else None
        _ptr(kappa)
        self._check(lib().clc_poisson_sht_batch(self.h, kp, P, nside, lmax, precision, pp, dd))
        return out

    def gal_trace(self, kappas, nside, lmax, chi, gz, gphi, gchi, precision=FP64, tape=True):
        """Galaxy shears gamma[2, ngal] through the planes kappas[N, Npix]
        (clc_gal_trace); returns (gamma, GalTape or None)."""
        N = kappas.shape[0]
        n = gz.numel()
        gamma = torch.empty(2, n, dtype=torch.float64, device=self.device)
        kp = (_p * N)(*[kappas[i].data_ptr() for i in range(N)])
        _ptr(kappas)
        ch = (_d * (N + 1))(*[float(c) for c in chi])
        h = _p()
        self._check(lib().clc_gal_trace(self.h, N, kp, nside, lmax, precision, ch, n, _ptr(gz), _ptr(gphi),
                                        _ptr(gchi), _ptr(gamma), ctypes.byref(h) if tape else None))
        return gamma, (GalTape(self, h, kappas) if tape else None)

    def gal_trace_mg(self, kappas, nside, params, chi, gz, gphi, gchi, tape=True):
        """Galaxy shears gamma[2, ngal] through SHT+MG planes kappas[N, Npix]
        (clc_gal_trace_mg, FP64 MG parameters); returns (gamma, GalTape or None)."""
        N = kappas.shape[0]
        n = gz.numel()
        gamma = torch.empty(2, n, dtype=torch.float64, device=self.device)
        kp = (_p * N)(*[kappas[i].data_ptr() for i in range(N)])
        _ptr(kappas)
        ch = (_d * (N + 1))(*[float(c) for c in chi])
        h = _p()
        self._check(lib().clc_gal_trace_mg(self.h, N, kp, nside, ctypes.byref(params), ch, n, _ptr(gz), _ptr(gphi),
                                           _ptr(gchi), _ptr(gamma), ctypes.byref(h) if tape else None))
        return gamma, (GalTape(self, h, kappas) if tape else None)

    def sht_plan(self, nsides, lmaxs, derivatives=True, graph=True, tune=False):
        return ShtPlan(self, nsides, lmaxs, derivatives, graph, tune)

    def gemm_f16x3(self, a_hi, a_lo, b_hi, b_lo):
        """d[b] = a_hi b_hi^T + a_hi b_lo^T + a_lo b_hi^T (tcgen05, FP32 accumulate)."""
        batch, M, K = a_hi.shape
        N = b_hi.shape[1]
        d = torch.empty(batch, M, N, dtype=torch.float32, device=self.device)
        self._check(lib().clc_gemm_f16x3(self.h, _ptr(a_hi), _ptr(a_lo), _ptr(b_hi), _ptr(b_lo), M, N, K, batch,
                                         _ptr(d)))
        return d

    def eb_analysis(self, g1, g2, nside, lmax):
        n = (lmax + 1) * (lmax + 2) // 2
        E = torch.empty(n, dtype=torch.complex128, device=self.device)
        B = torch.empty(n, dtype=torch.complex128, device=self.device)
        self._check(lib().clc_eb_analysis(self.h, _ptr(g1), _ptr(g2), nside, lmax, _ptr(E), _ptr(B)))
        return E, B

    def power_spectrum(self, alm, lmax, alm2=None):
        cl = torch.empty(lmax + 1, dtype=torch.float64, device=self.device)
        self._check(lib().clc_power_spectrum(self.h, _ptr(alm), _ptr(alm2), lmax, _ptr(cl)))
        return cl

    def lensing_spectra(self, A, nside, lmax, x=None):
        """dict of C_l for kappa, E, B, omega from A[4, 12 nside^2] (rays from
        the RING pixel centres); x[3, 12 nside^2]: the rays' source positions,
        whose basis A is in (None: A is in the pixel basis)."""
        cl = torch.empty(4, lmax + 1, dtype=torch.float64, device=self.device)
        self._check(lib().clc_lensing_spectra(self.h, _ptr(x), _ptr(A), nside, lmax, _ptr(cl)))
        return dict(zip(("kappa", "E", "B", "omega"), cl))

    # -- step 3 / 4 ---------------------------------------------------------
    def solution(self, nside_fine, params, domain=None):
        """A plane's multigrid state; domain: NEST bundle indices of a partial
        sky (None: every bundle)."""
        return Solution(self, nside_fine, params, domain)

    def poisson_shtmg(self, kappa_fine, nside_fine, sol, derivatives=False, check=True):
        npx = 12 * nside_fine * nside_fine
        out, d = self._derivs(npx, ("a_th", "a_ph", "u_tt", "u_pp", "u_tp") if derivatives else ())
        rc = lib().clc_poisson_shtmg(self.h, _ptr(kappa_fine), nside_fine, ctypes.byref(sol.params), sol.h,
                                     ctypes.byref(d) if derivatives else None)
        if rc != OK and not (rc == ENOTCONVERGED and not check):
            self._check(rc)
        return out

    def lens_derivs(self, sol, z, phi, bundle=None):
        out, d = self._derivs(z.numel(), ("a_th", "a_ph", "u_tt", "u_pp", "u_tp"))
        self._check(lib().clc_lens_derivs(self.h, sol.h, _ptr(z), _ptr(phi), _ptr(bundle), z.numel(), ctypes.byref(d)))
        return out

    # -- step 5 -------------------------------------------------------------
    def rays(self, n):
        return RayState(self, n)

    def rays_init(self, rays, z, phi, chi0, nside_bundle=0):
        self._check(lib().clc_rays_init(self.h, _ptr(z), _ptr(phi), float(chi0), int(nside_bundle),
                                        ctypes.byref(rays.struct())))

    def rays_init_pixels(self, rays, nside, chi0, nside_bundle=0):
        self._check(lib().clc_rays_init_pixels(self.h, int(nside), float(chi0), int(nside_bundle),
                                               ctypes.byref(rays.struct())))

    def ray_step(self, rays, chi_prev, chi_n, chi_next, sol=None, maps=None, nside_maps=0):
        d = None
        if maps is not None:
            d = Derivs(*[_ptr(maps[k]) for k in ("a_th", "a_ph", "u_tt", "u_pp", "u_tp")])
        self._check(lib().clc_ray_step(self.h, sol.h if sol is not None else None,
                                       ctypes.byref(d) if d is not None else None, int(nside_maps),
                                       float(chi_prev), float(chi_n), float(chi_next), ctypes.byref(rays.struct())))

    def find_images(self, nside, x, A, g, max_images=4, matrices=True):
        """Images of galaxies at source positions g [3, M] from rays started at
        the RING pixel centres of nside with source positions x [3, npix] and
        matrices A [4, npix].  Returns (nimg [M] int32, tri [max_images, M]
        int64, img [3, max_images, M] unit vectors, A_img [4, max_images, M]
        or None)."""
        M = g.shape[-1]
        dev = self.device
        nimg = torch.empty(M, dtype=torch.int32, device=dev)
        tri = torch.empty(max_images, M, dtype=torch.int64, device=dev)
        img = torch.empty(3, max_images, M, dtype=torch.float64, device=dev)
        Ai = torch.empty(4, max_images, M, dtype=torch.float64, device=dev) if matrices else None
        self._check(lib().clc_find_images(self.h, int(nside), _ptr(x), _ptr(A) if matrices else None, int(M),
                                          _ptr(g), int(max_images), _ptr(nimg), _ptr(tri), _ptr(img), _ptr(Ai)))
        return nimg, tri, img, Ai

    def raytrace_planes(self, solver, params, kappa_planes, nside, chi, rays):
        n = len(kappa_planes)
        arr = (ctypes.c_void_p * n)(*[k.data_ptr() for k in kappa_planes])
        chis = (ctypes.c_double * len(chi))(*[float(c) for c in chi])
        self._check(lib().clc_raytrace_planes(self.h, solver, ctypes.byref(params), arr, n, nside, chis,
                                              ctypes.byref(rays.struct())))


class Solution:
    """Multigrid state of one plane (clc_plane_solution)."""

    def __init__(self, ctx, nside_fine, params, domain=None):
        self.ctx = ctx
        self.params = params
        self.nside_fine = nside_fine
        h = ctypes.c_void_p()
        if domain is None:
            ctx._check(lib().clc_solution_create(ctx.h, nside_fine, ctypes.byref(params), ctypes.byref(h)))
        else:
            d = [int(b) for b in domain]
            arr = (ctypes.c_int32 * len(d))(*d)
            ctx._check(lib().clc_solution_create_domain(ctx.h, nside_fine, ctypes.byref(params), arr, len(d),
                                                        ctypes.byref(h)))
        self.h = h

    def domain(self):
        """(number of patches, lookups outside the domain since the last solve)."""
        n = _i()
        o = _i64()
        self.ctx._check(lib().clc_solution_domain(self.h, ctypes.byref(n), ctypes.byref(o)))
        return n.value, o.value

    def info(self):
        c = ctypes.c_int()
        r = ctypes.c_double()
        lib().clc_solution_info(self.h, ctypes.byref(c), ctypes.byref(r))
        return c.value, r.value

    def close(self):
        if getattr(self, "h", None):
            self.ctx.sync()
            lib().clc_solution_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RayState:
    """Device ray state in the library's SoA layout."""

    def __init__(self, ctx, n):
        dev = ctx.device
        self.n = n
        self.x = torch.empty(3, n, dtype=torch.float64, device=dev)
        self.beta = torch.empty(3, n, dtype=torch.float64, device=dev)
        self.A = torch.empty(4, n, dtype=torch.float64, device=dev)
        self.Ap = torch.empty(4, n, dtype=torch.float64, device=dev)
        self.bundle = torch.zeros(n, dtype=torch.int32, device=dev)

    def struct(self):
        return Rays(self.n, _ptr(self.x), _ptr(self.beta), _ptr(self.A), _ptr(self.Ap), _ptr(self.bundle))


class GalTape:
    """Checkpoints of one clc_gal_trace for its adjoint."""

    def __init__(self, ctx, h, kappas):
        self.ctx, self.h, self.kappas = ctx, h, kappas

    def adjoint(self, gamma_bar):
        kb = torch.empty_like(self.kappas)
        N = kb.shape[0]
        ptrs = (_p * N)(*[kb[i].data_ptr() for i in range(N)])
        self.ctx._check(lib().clc_gal_trace_adjoint(self.h, _ptr(gamma_bar.contiguous()), ptrs))
        return kb

    def close(self):
        if self.h:
            lib().clc_gal_tape_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GalaxyShear(torch.autograd.Function):
    """gamma[2, ngal] = galaxy shears through the planes kappas[N, Npix], each
    solved by the pure SHT (lmax_or_params an int band limit) or by SHT+MG
    (lmax_or_params an FP64 mg_params); the backward pass is the library's
    adjoint (checkpointed ray states, recomputed planes, the transposed SHT
    and, for SHT+MG, the adjoint patch solve)."""

    @staticmethod
    def forward(fctx, kappas, lib_ctx, nside, lmax_or_params, chi, gz, gphi, gchi, precision):
        k = kappas.detach().contiguous()
        if isinstance(lmax_or_params, MGParams):
            gamma, tape = lib_ctx.gal_trace_mg(k, nside, lmax_or_params, chi, gz, gphi, gchi)
        else:
            gamma, tape = lib_ctx.gal_trace(k, nside, lmax_or_params, chi, gz, gphi, gchi, precision)
        fctx.tape = tape
        return gamma

    @staticmethod
    def backward(fctx, gbar):
        kb = fctx.tape.adjoint(gbar)
        fctx.tape.close()
        return kb, None, None, None, None, None, None, None, None


def galaxy_shear(lib_ctx, kappas, nside, lmax, chi, gz, gphi, gchi, precision=FP64):
    """Differentiable galaxy shears (see GalaxyShear); lmax may be an
    mg_params (FP64) for the SHT+MG solver."""
    return GalaxyShear.apply(kappas, lib_ctx, nside, lmax, chi, gz, gphi, gchi, precision)


class ShtPlan:
    """clc_sht_plan: a fixed batch of mixed-precision pure-SHT plane solves of
    mixed (nside, lmax), optionally replayed as a CUDA graph and autotuned."""

    def __init__(self, ctx, nsides, lmaxs, derivatives=True, graph=True, tune=False):
        self.ctx = ctx
        self.nsides = [int(v) for v in nsides]
        self.lmaxs = [int(v) for v in lmaxs]
        self.derivatives = derivatives
        n = len(self.nsides)
        h = _p()
        ns = (_i * n)(*self.nsides)
        lm = (_i * n)(*self.lmaxs)
        flags = (PLAN_GRAPH if graph else 0) | (PLAN_TUNE if tune else 0)
        ctx._check(lib().clc_sht_plan_create(ctx.h, n, ns, lm, 1 if derivatives else 0, flags, ctypes.byref(h)))
        self.h = h

    def execute(self, kappas, outputs):
        """kappas: list of device maps; outputs: list of dicts with 'psi' and,
        for a plan with derivatives, 'a_th', 'a_ph', 'u_tt', 'u_pp', 'u_tp'."""
        n = len(self.nsides)
        kp = (_p * n)(*[_ptr(k) for k in kappas])
        pp = (_p * n)(*[_ptr(o.get("psi")) for o in outputs])
        dd = None
        if self.derivatives:
            dd = (Derivs * n)(*[Derivs(*[_ptr(o.get(k)) for k in ("a_th", "a_ph", "u_tt", "u_pp", "u_tp")])
                                for o in outputs])
        self.ctx._check(lib().clc_sht_plan_execute(self.h, kp, pp, dd))

    def info(self):
        shape = (_i * 5)()
        ms = (_d * 6)()
        nb = ctypes.c_size_t()
        self.ctx._check(lib().clc_sht_plan_info(self.h, shape, ms, ctypes.byref(nb)))
        return {"shape": list(shape), "stage_ms": list(ms), "device_bytes": nb.value}

    def close(self):
        if self.h:
            lib().clc_sht_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_params(nside_sht, lmax, nside_bundle, ncell=256, nu1=2, nu2=2, max_cycles=60, fixed_cycles=0, tol=1e-10,
              precision=FP64, stop_rule=STOP_RESIDUAL, eps=0.1, refine_cycles=0):
    return MGParams(nside_sht, lmax, nside_bundle, ncell, nu1, nu2, max_cycles, fixed_cycles, tol, precision,
                    stop_rule, eps, refine_cycles)
