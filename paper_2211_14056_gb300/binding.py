"""ctypes binding of include/madflow_gb300.h (argument marshalling only).

Every computation runs in the CUDA library; these wrappers check Python-side
arguments (dtype, device, size, contiguity of torch tensors), pass raw
pointers and the current CUDA stream, and turn negative status codes into
``MFError`` carrying ``mf_last_error()``.  Loading fails loudly if the library
has not been built.
"""
import ctypes as C
import functools
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "lib", "libmadflow_gb300.so")

MF_OK, MF_ERR_ARG, MF_ERR_CUDA, MF_ERR_UNSUPPORTED, MF_ERR_COLOUR, MF_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
MF_WARN_NEWTON, MF_WARN_CAPACITY = 1, 2
MF_PROC_GG_TTX, MF_PROC_GG_TTXG, MF_PROC_GG_TTXGG, MF_PROC_UUX_TTXGG, MF_PROC_EE_MUMU = 1, 2, 3, 4, 5
MF_PROC_UXU_TTXGG, MF_PROC_UG_TTXGU, MF_PROC_GU_TTXGU, MF_PROC_UXG_TTXGUX, MF_PROC_GUX_TTXGUX = 6, 7, 8, 9, 10
MF_FP64, MF_FP32, MF_FP32_TC = 0, 1, 2

_NGLUON = {MF_PROC_GG_TTX: 2, MF_PROC_GG_TTXG: 3, MF_PROC_GG_TTXGG: 4, MF_PROC_UUX_TTXGG: 4, MF_PROC_EE_MUMU: 2,
           MF_PROC_UXU_TTXGG: 4, MF_PROC_UG_TTXGU: 4, MF_PROC_GU_TTXGU: 4, MF_PROC_UXG_TTXGUX: 4,
           MF_PROC_GUX_TTXGUX: 4}
_TWO_QUARK_LINES = {MF_PROC_UUX_TTXGG, MF_PROC_UXU_TTXGG, MF_PROC_UG_TTXGU, MF_PROC_GU_TTXGU, MF_PROC_UXG_TTXGUX,
                    MF_PROC_GUX_TTXGUX}
ALPHA_EM = 1.0 / 137.035999     # Thomson limit; e = sqrt(4 pi alpha)


class MFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


class ProcessDesc(C.Structure):
    _fields_ = [
        ("process_id", C.c_int), ("n_ext", C.c_int), ("masses", C.POINTER(C.c_double)),
        ("top_width", C.c_double), ("g_s", C.c_double), ("n_flow", C.c_int),
        ("colour_num", C.POINTER(C.c_int64)), ("colour_den", C.c_int64), ("sqrt_s", C.c_double),
        ("lumi", C.c_int), ("lumi_N", C.c_double), ("lumi_a", C.c_double), ("lumi_b", C.c_double),
        ("pt_cut_g", C.c_double), ("dr_cut_gg", C.c_double), ("precision", C.c_int),
        ("e_qed", C.c_double), ("pdf", C.c_void_p), ("n_pairs", C.c_int), ("pairs", C.POINTER(C.c_int)),
        ("mu_f", C.c_double),
    ]


class Result(C.Structure):
    _fields_ = [
        ("I_k", C.c_double), ("sigma_k", C.c_double), ("I", C.c_double), ("sigma", C.c_double),
        ("chi2dof", C.c_double), ("n_events", C.c_int64), ("n_pass", C.c_int64),
        ("n_newton_fail", C.c_int64), ("iterations", C.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = {
    "mf_init_process": (C.c_int, [C.POINTER(ProcessDesc), C.POINTER(C.c_void_p)]),
    "mf_destroy_process": (C.c_int, [C.c_void_p]),
    "mf_process_ndim": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "mf_set_ctas_per_sm": (C.c_int, [C.c_void_p, C.c_int]),
    "mf_set_launch_shape": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "mf_grid_create": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "mf_grid_destroy": (C.c_int, [C.c_void_p]),
    "mf_grid_get": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mf_grid_set": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mf_grid_reset": (C.c_int, [C.c_void_p]),
    "mf_grid_history": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_void_p, C.c_void_p]),
    "mf_grid_set_history": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mf_sample": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.c_int64, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_void_p]),
    "mf_matrix_element": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mf_matrix_element_hel": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mf_set_helicity_sampling": (C.c_int, [C.c_void_p, C.c_int]),
    "mf_grid_helicity": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int]),
    "mf_grid_set_helicity": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int]),
    "mf_uniforms": (C.c_int, [C.c_uint64, C.c_int, C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    "mf_vegas_iterate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.c_int64, C.c_int,
                                   C.POINTER(Result), C.c_void_p, C.c_void_p]),
    "mf_vegas_accumulate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.c_int64, C.c_int64,
                                      C.c_void_p, C.c_void_p]),
    "mf_grid_totals": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int)]),
    "mf_vegas_finish": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.POINTER(Result), C.c_void_p]),
    "mf_fma_throughput": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "mf_unweight": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.c_int64, C.c_int64, C.c_double,
                              C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64),
                              C.POINTER(C.c_int64), C.c_void_p]),
    "mf_grid_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "mf_grid_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "mf_vegas_accumulate_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_uint64, C.c_int, C.c_int64,
                                             C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mf_mixed_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_int,
                                  C.POINTER(C.c_void_p)]),
    "mf_mixed_destroy": (C.c_int, [C.c_void_p]),
    "mf_mixed_run": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.c_int, C.POINTER(Result), C.c_void_p]),
    "mf_mixed_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mf_mixed_use_graph": (C.c_int, [C.c_void_p, C.c_int]),
    "mf_mixed_autotune": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                    C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p]),
    "mf_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.c_int64, C.POINTER(C.c_double),
                          C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_void_p]),
    "mf_grad_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.c_int64, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_void_p]),
    "mf_pdf_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                C.POINTER(C.c_double), C.POINTER(C.c_void_p)]),
    "mf_pdf_destroy": (C.c_int, [C.c_void_p]),
    "mf_pdf_eval": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p]),
    "mf_last_error": (C.c_char_p, []),
    "mf_kernel_launches": (C.c_int64, []),
}


def library_path():
    return _LIB_PATH


@functools.lru_cache(maxsize=None)
def load_library():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with `python -m paper_2211_14056_gb300.build` "
                          "(there is no CPU fallback)")
    lib = C.CDLL(_LIB_PATH)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _check(st, allow_warn=True):
    if st < 0 or (st > 0 and not allow_warn):
        raise MFError(st, load_library().mf_last_error().decode())
    return st


def kernel_launches():
    return int(load_library().mf_kernel_launches())


def fma_throughput(precision):
    """Measured FMA-pipe throughput of the current device, TFLOP/s."""
    t = C.c_double()
    _check(load_library().mf_fma_throughput(precision, C.byref(t)))
    return t.value


def uniforms(seed, it, n, ndim, first_event=0, out=None, stream=None):
    """The Philox uniforms y[ndim, n] (float64, device) of global events
    first_event .. first_event + n - 1 of iteration `it` (mf_uniforms)."""
    import torch
    if out is None:
        out = torch.empty((ndim, n), dtype=torch.float64, device="cuda")
    _check(load_library().mf_uniforms(seed, it, first_event, n, ndim, _ptr(out, torch.float64, ndim * n, "y"),
                                      _stream(stream)))
    return out


@functools.lru_cache(maxsize=None)
def colour_matrix(ngluons):
    """(integer numerators [n!*n!], denominator) of the trace-basis colour matrix."""
    from .gen_tables import colour_matrix_exact
    _, M, D = colour_matrix_exact(ngluons)
    return [x for row in M for x in row], D


@functools.lru_cache(maxsize=None)
def colour_matrix_uux():
    """(integer numerators [12*12], denominator) of the u u~ -> t t~ g g colour matrix."""
    from .gen_uux import colour_matrix_exact
    M, D = colour_matrix_exact()
    return [x for row in M for x in row], D


def _ptr(t, dtype, numel, name):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous CUDA tensor of {dtype}")
    if t.numel() < numel:
        raise ValueError(f"{name}: need at least {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _refine_bits(refine):
    """refine as the C mask: True -> edges and helicity table (1 | 2), False ->
    nothing, "edges" -> 1, "helicities" -> 2, or the mask itself."""
    if refine is True:
        return 3
    if refine is False or refine is None:
        return 0
    if refine == "edges":
        return 1
    if refine == "helicities":
        return 2
    return int(refine)


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class PDFSet:
    """A tabulated parton-density set loaded on the device (mf_pdf_create):
    xf [nflav][nq][nx] = x f(x, Q^2) on nodes uniform in ln x and ln Q^2."""

    def __init__(self, x_min, x_max, q2_min, q2_max, xf):
        import numpy as np
        t = np.ascontiguousarray(xf, dtype=np.float64)
        if t.ndim != 3:
            raise ValueError("xf must be [nflav][nq][nx]")
        self.nflav, self.nq, self.nx = t.shape
        h = C.c_void_p()
        _check(load_library().mf_pdf_create(self.nflav, self.nq, self.nx, x_min, x_max, q2_min, q2_max,
                                            t.ctypes.data_as(C.POINTER(C.c_double)), C.byref(h)))
        self._h = h

    @classmethod
    def from_dict(cls, d):
        return cls(d["x_min"], d["x_max"], d["q2_min"], d["q2_max"], d["xf"])

    def close(self):
        if getattr(self, "_h", None):
            load_library().mf_pdf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eval(self, flavour, n, x, q2, out, precision=MF_FP64, stream=None):
        """out[e] = x f(x[e], q2[e]) of one flavour (device float64 tensors)."""
        import torch
        _check(load_library().mf_pdf_eval(self._h, precision, flavour, n, _ptr(x, torch.float64, n, "x"),
                                          _ptr(q2, torch.float64, n, "q2"), _ptr(out, torch.float64, n, "xf"),
                                          _stream(stream)))


class Process:
    """A configured process (mf_init_process) and its launches.  lumi: False
    (fixed partonic energy), True (synthetic gluon luminosity) or "pdf"
    (tabulated densities: pdf = a PDFSet, pairs = [(flavour a, flavour b)...],
    mu_f = factorisation scale over sqrt(s_hat))."""

    def __init__(self, process_id, mt=173.0, wt=0.0, gs=1.2177, sqrt_s=1000.0, lumi=False,
                 lumi_N=1.0, lumi_a=-1.1, lumi_b=5.0, pt_cut=0.0, dr_cut=0.0, precision=MF_FP64,
                 colour=None, e_qed=None, masses=None, pdf=None, pairs=None, mu_f=0.5):
        lib = load_library()
        ng = _NGLUON.get(process_id)
        if ng is None:
            raise MFError(MF_ERR_UNSUPPORTED, "unknown process id")
        self.ngluons, self.n_ext = ng, ng + 2
        self.process_id = process_id
        if masses is None:
            masses = [0.0] * 4 if process_id == MF_PROC_EE_MUMU else [0.0, 0.0, mt, mt] + [0.0] * (ng - 2)
        masses = (C.c_double * self.n_ext)(*masses)
        if e_qed is None:
            e_qed = math.sqrt(4 * math.pi * ALPHA_EM)
        if process_id == MF_PROC_EE_MUMU:
            num, den = colour if colour is not None else ([1], 1)
            nflow = 1
        elif process_id in _TWO_QUARK_LINES:
            num, den = colour if colour is not None else colour_matrix_uux()
            nflow = 12
        else:
            num, den = colour if colour is not None else colour_matrix(ng)
            nflow = math.factorial(ng)
        cnum = (C.c_int64 * len(num))(*num)
        lumi_code = 2 if lumi == "pdf" else (1 if lumi else 0)
        pdf_h, npairs, cpairs = None, 0, None
        if lumi_code == 2:
            if pdf is None or not pairs:
                raise ValueError('lumi="pdf" needs pdf (a PDFSet) and pairs')
            flat = [int(f) for ab in pairs for f in ab]
            npairs, cpairs = len(pairs), (C.c_int * len(flat))(*flat)
            pdf_h = pdf._h
            self._pdf = pdf                    # the set must outlive the process
        d = ProcessDesc(process_id, self.n_ext, masses, wt, gs, nflow, cnum, den, sqrt_s,
                        lumi_code, lumi_N, lumi_a, lumi_b, pt_cut, dr_cut, precision, e_qed, pdf_h, npairs,
                        cpairs, mu_f)
        h = C.c_void_p()
        _check(lib.mf_init_process(C.byref(d), C.byref(h)))
        self._h = h
        nd = C.c_int()
        _check(lib.mf_process_ndim(h, C.byref(nd)))
        self.ndim = nd.value
        self.precision = precision

    def close(self):
        if getattr(self, "_h", None):
            load_library().mf_destroy_process(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_ctas_per_sm(self, c):
        _check(load_library().mf_set_ctas_per_sm(self._h, int(c)))

    def set_launch_shape(self, warps_per_cta):
        """Warps per CTA of the iteration's |M|^2 kernel (0: default); returns
        how many such CTAs fit on one SM."""
        c = C.c_int()
        _check(load_library().mf_set_launch_shape(self._h, int(warps_per_cta), C.byref(c)))
        return c.value

    def grid(self, nbins=50):
        return Grid(self, nbins)

    def sample(self, grid, seed, it, n, momenta=None, weight_ps=None, bins=None, stream=None):
        import torch
        p = _ptr(momenta, torch.float64, self.n_ext * 4 * n, "momenta")
        w = _ptr(weight_ps, torch.float64, n, "weight_ps")
        b = _ptr(bins, torch.uint8, self.ndim * n, "bins")
        _check(load_library().mf_sample(self._h, grid._h, seed, it, n, p, w, b, _stream(stream)))

    def matrix_element(self, n, momenta, me2, stream=None):
        import torch
        _check(load_library().mf_matrix_element(
            self._h, n, _ptr(momenta, torch.float64, self.n_ext * 4 * n, "momenta"),
            _ptr(me2, torch.float64, n, "me2"), _stream(stream)))

    def matrix_element_hel(self, n, momenta, hel, me2, stream=None):
        """|M|^2 of one helicity configuration per event (hel: int32 [n], bit
        g: gluon g helicity +1, bit NG: antitop helicity +1; the top summed)."""
        import torch
        _check(load_library().mf_matrix_element_hel(
            self._h, n, _ptr(momenta, torch.float64, self.n_ext * 4 * n, "momenta"),
            _ptr(hel, torch.int32, n, "hel"), _ptr(me2, torch.float64, n, "me2"), _stream(stream)))

    def set_helicity_sampling(self, on):
        """Iterations estimate |M|^2 from one helicity configuration per event
        drawn from the grid's table (True), also adapting that table as the
        grid refines ("adaptive"), or sum the helicities (False, the default)."""
        mode = 2 if on == "adaptive" else (1 if on else 0)
        _check(load_library().mf_set_helicity_sampling(self._h, mode))

    def vegas_iterate(self, grid, seed, it, n, refine=True, weights=None, stream=None):
        import torch
        r = Result()
        st = _check(load_library().mf_vegas_iterate(
            self._h, grid._h, seed, it, n, _refine_bits(refine), C.byref(r),
            _ptr(weights, torch.float64, n, "weights"), _stream(stream)))
        out = r.as_dict()
        out["status"] = st
        return out

    def vegas_accumulate(self, grid, seed, it, first_event, n, weights=None, stream=None):
        import torch
        _check(load_library().mf_vegas_accumulate(
            self._h, grid._h, seed, it, first_event, n, _ptr(weights, torch.float64, n, "weights"),
            _stream(stream)))

    def vegas_accumulate_static(self, edges, nbins, seed, it, first_event, n, totals, weights=None, stream=None):
        """Allocation-free accumulation into caller-owned device buffers."""
        import torch
        _check(load_library().mf_vegas_accumulate_static(
            self._h, _ptr(edges, torch.float64, self.ndim * (nbins + 1), "edges"), nbins, seed, it, first_event, n,
            _ptr(totals, torch.float64, 2 + self.ndim * nbins + 2, "totals"),
            _ptr(weights, torch.float64, n, "weights"), _stream(stream)))

    def unweight(self, grid, seed, it, first_event, n, w_max, capacity, momenta=None, weight=None, event=None,
                 stream=None):
        """Hit-or-miss unweighting (mf_unweight) of events first_event ..
        first_event + n - 1 into caller-owned device buffers (momenta float64
        [n_ext*4*capacity], weight float64 [capacity], event int64
        [capacity]); returns (kept, overweight, status)."""
        import torch
        k, o = C.c_int64(), C.c_int64()
        st = _check(load_library().mf_unweight(
            self._h, grid._h, seed, it, first_event, n, w_max, capacity,
            _ptr(momenta, torch.float64, self.n_ext * 4 * capacity, "momenta"),
            _ptr(weight, torch.float64, capacity, "weight"), _ptr(event, torch.int64, capacity, "event"),
            C.byref(k), C.byref(o), _stream(stream)))
        return k.value, o.value, st

    def grad(self, grid, seed, it, n, dw_dtheta=None, dw_dy=None, stream=None, forward=False):
        """sigma and [dsigma/dg_s, dsigma/dm_t, dsigma/dGamma_t] of iteration `it`
        over events 0..n-1 (mf_grad, reverse mode; mf_grad_forward with
        forward=True); the optional device tensors receive the per-event
        derivatives ([3, n] and [ndim, n], float64)."""
        import torch
        sig = C.c_double()
        ds = (C.c_double * 3)()
        fn = load_library().mf_grad_forward if forward else load_library().mf_grad
        _check(fn(
            self._h, grid._h, seed, it, n, C.byref(sig), ds,
            _ptr(dw_dtheta, torch.float64, 3 * n, "dw_dtheta"), _ptr(dw_dy, torch.float64, self.ndim * n, "dw_dy"),
            _stream(stream)))
        return sig.value, [ds[0], ds[1], ds[2]]

    def vegas_finish(self, grid, n_total, refine=True, stream=None):
        r = Result()
        st = _check(load_library().mf_vegas_finish(self._h, grid._h, n_total, _refine_bits(refine), C.byref(r),
                                                   _stream(stream)))
        out = r.as_dict()
        out["status"] = st
        return out


class Grid:
    """A Vegas grid (mf_grid_create) bound to a process."""

    def __init__(self, proc, nbins=50):
        self.proc, self.nbins, self.ndim = proc, nbins, proc.ndim
        # helicity configurations of the table (gluon-initiated processes:
        # 2^(NG+1); two-quark-line ones: 32; e+ e- -> mu+ mu-: none)
        if proc.process_id in (MF_PROC_GG_TTX, MF_PROC_GG_TTXG, MF_PROC_GG_TTXGG):
            self.n_configs = 1 << (proc.n_ext - 1)
        elif proc.process_id == MF_PROC_EE_MUMU:
            self.n_configs = 0
        else:
            self.n_configs = 32
        h = C.c_void_p()
        _check(load_library().mf_grid_create(proc._h, nbins, C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load_library().mf_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        import numpy as np
        out = np.empty((self.ndim, self.nbins + 1))
        _check(load_library().mf_grid_get(self._h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def set(self, edges):
        import numpy as np
        e = np.ascontiguousarray(edges, dtype=np.float64)
        if e.shape != (self.ndim, self.nbins + 1):
            raise ValueError(f"edges must have shape {(self.ndim, self.nbins + 1)}")
        _check(load_library().mf_grid_set(self._h, e.ctypes.data_as(C.POINTER(C.c_double))))

    def reset(self):
        _check(load_library().mf_grid_reset(self._h))

    def history(self):
        """(I_k, sigma_k^2) of the recorded iterations, as numpy arrays."""
        import numpy as np
        n = C.c_int(0)
        _check(load_library().mf_grid_history(self._h, C.byref(n), None, None))
        I = np.zeros(max(n.value, 1))
        v = np.zeros(max(n.value, 1))
        _check(load_library().mf_grid_history(self._h, C.byref(n), I.ctypes.data, v.ctypes.data))
        return I[:n.value], v[:n.value]

    def helicity(self):
        """Probabilities of the helicity table (2^(NG+1) configurations), or
        None for a process without one."""
        import numpy as np
        if self.n_configs == 0:
            return None
        out = np.empty(self.n_configs)
        _check(load_library().mf_grid_helicity(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), self.n_configs))
        return out

    def set_helicity(self, prob):
        import numpy as np
        p = np.ascontiguousarray(prob, dtype=np.float64)
        _check(load_library().mf_grid_set_helicity(self._h, p.ctypes.data_as(C.POINTER(C.c_double)), p.size))

    def checkpoint(self):
        """The grid's whole state: edges, the helicity table and the recorded
        iterations."""
        I, v = self.history()
        return {"edges": self.get(), "I_k": I, "var_k": v, "helicity": self.helicity()}

    def restore(self, state):
        import numpy as np
        self.set(state["edges"])
        if state.get("helicity") is not None:
            self.set_helicity(state["helicity"])
        I = np.ascontiguousarray(state["I_k"], dtype=np.float64)
        v = np.ascontiguousarray(state["var_k"], dtype=np.float64)
        if I.shape != v.shape or I.ndim != 1:
            raise ValueError("I_k and var_k must be 1-D arrays of one length")
        _check(load_library().mf_grid_set_history(self._h, int(I.size), I.ctypes.data if I.size else None,
                                                  v.ctypes.data if v.size else None))

    def profile(self, enable=True):
        _check(load_library().mf_grid_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """(sampling ms, |M|^2 ms, chunks) of the last accumulation."""
        a, b, c = C.c_double(), C.c_double(), C.c_int()
        _check(load_library().mf_grid_profile_read(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def totals(self):
        """(device address, length) of the accumulated totals (double[length])."""
        ptr, cnt = C.c_void_p(), C.c_int()
        _check(load_library().mf_grid_totals(self._h, C.byref(ptr), C.byref(cnt)))
        return ptr.value, cnt.value


class Mixed:
    """Several processes in one iteration (mf_mixed_*): one sampling launch,
    one persistent |M|^2 launch with a cost-ordered work queue."""

    def __init__(self, procs, grids, n):
        k = len(procs)
        self.procs, self.grids, self.n = list(procs), list(grids), list(n)
        ph = (C.c_void_p * k)(*[p._h.value for p in procs])
        gh = (C.c_void_p * k)(*[g._h.value for g in grids])
        nn = (C.c_int64 * k)(*n)
        h = C.c_void_p()
        _check(load_library().mf_mixed_create(ph, gh, nn, k, C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load_library().mf_mixed_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, seed, it, refine=True, stream=None):
        out = (Result * len(self.procs))()
        st = _check(load_library().mf_mixed_run(self._h, seed, it, 1 if refine else 0, out, _stream(stream)))
        res = [r.as_dict() for r in out]
        for r in res:
            r["status"] = st
        return res

    def set_launch(self, ctas_per_sm, tile):
        _check(load_library().mf_mixed_set_launch(self._h, ctas_per_sm, tile))

    def use_graph(self, enable=True):
        _check(load_library().mf_mixed_use_graph(self._h, 1 if enable else 0))

    def autotune(self, seed, candidates, stream=None):
        """candidates: list of (ctas_per_sm, tile); returns (times_ms, best index)."""
        k = len(candidates)
        cc = (C.c_int * k)(*[c for c, _ in candidates])
        ct = (C.c_int * k)(*[t for _, t in candidates])
        ms = (C.c_double * k)()
        best = C.c_int()
        _check(load_library().mf_mixed_autotune(self._h, seed, k, cc, ct, ms, C.byref(best), _stream(stream)))
        return list(ms), best.value
