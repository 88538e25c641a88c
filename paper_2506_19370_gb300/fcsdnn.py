"""Python binding of libfcsdnn (C ABI in include/fcsdnn.h): argument marshalling only.

Every step of the FC-SDNN stage runs in the CUDA library; this module loads it
with ctypes, fills the descriptor structs, passes device pointers of torch
tensors and converts between per-patch arrays and the library's flat layouts.
It raises if the library is missing: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfcsdnn.so")

F32, F64 = 0, 1
N_PARAMS = 1732
ERRORS = {0: "ok", -1: "EINVAL", -2: "EOVERLAP", -3: "EUNSUPPORTED", -4: "ECUDA", -5: "ENOMEM",
          -6: "ENONFINITE", -7: "ENEGATIVE", -8: "ESCRATCH"}
NOALLOC_BATCH_MAX = 4096

# every entry point of include/fcsdnn.h
EXPORTS = ("fcs_default_options", "fc_setup", "fc_destroy", "fcs_get_layout", "fcs_build_table", "fcs_line_c",
           "fc_derivative", "euler_rhs", "rk_stage", "patch_exchange", "fcs_time_step", "fcs_conservation_sums",
           "sdnn_set_weights", "sdnn_get_weights", "sdnn_classify", "sdnn_indicator", "av_assemble",
           "sdnn_train_step", "sdnn_gradient", "sdnn_gradient_noalloc", "fcs_step", "fcs_step_graph", "fcs_status",
           "fcs_strerror", "fcs_filter", "fcs_smear_initial", "fcs_alu_probe", "sdnn_windows")


class FcsError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {ERRORS.get(code, code)}")
        self.code = code


class PatchDesc(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("bc", ctypes.c_int * 4), ("cartesian", ctypes.c_int),
                ("box", ctypes.c_double * 4), ("x", ctypes.POINTER(ctypes.c_double)),
                ("y", ctypes.POINTER(ctypes.c_double)), ("lcut", ctypes.c_int * 2),
                ("inflow", ctypes.POINTER(ctypes.c_double))]


class Options(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("n_f", ctypes.c_int), ("dtype", ctypes.c_int),
                ("instances", ctypes.c_int), ("inflow", ctypes.c_double * 4), ("p_out", ctypes.c_double),
                ("c_mu", ctypes.c_double), ("av_radius", ctypes.c_int), ("c_policy", ctypes.c_int),
                ("train_batch_max", ctypes.c_int), ("autotune", ctypes.c_int), ("filter_alpha", ctypes.c_double),
                ("filter_p", ctypes.c_int), ("filter_step", ctypes.c_int), ("smear_p", ctypes.c_int),
                ("op_form", ctypes.c_int)]


class Layout(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int), ("npatch", ctypes.c_int), ("dtype", ctypes.c_int), ("d", ctypes.c_int),
                ("state_elems", ctypes.c_size_t), ("scalar_elems", ctypes.c_size_t), ("windows", ctypes.c_size_t),
                ("state_off", ctypes.POINTER(ctypes.c_int64)), ("scalar_off", ctypes.POINTER(ctypes.c_int64)),
                ("window_off", ctypes.POINTER(ctypes.c_int64)), ("tile_width", ctypes.c_int),
                ("launches_stage", ctypes.c_int), ("launches_stage_visc", ctypes.c_int),
                ("launches_exchange", ctypes.c_int), ("launches_av", ctypes.c_int)]


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfcsdnn.so not built ({LIB_PATH}); run paper_2506_19370_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "fcs_default_options": (None, [ctypes.POINTER(Options)]),
            "fc_setup": (i, [ctypes.POINTER(vp), i, i, ctypes.POINTER(PatchDesc), i, ctypes.POINTER(Options)]),
            "fc_destroy": (None, [vp]),
            "fcs_get_layout": (i, [vp, ctypes.POINTER(Layout)]),
            "fcs_build_table": (i, [i, i, ctypes.POINTER(ctypes.c_double)]),
            "fcs_line_c": (i, [vp, i]),
            "fc_derivative": (i, [vp, vp, vp, i, i, vp]),
            "euler_rhs": (i, [vp, vp, vp, vp, vp]),
            "rk_stage": (i, [vp, i, d, vp, vp, vp, vp, vp, vp, vp]),
            "patch_exchange": (i, [vp, vp, i, vp]),
            "fcs_time_step": (i, [vp, vp, vp, vp, vp]),
            "fcs_conservation_sums": (i, [vp, vp, vp, vp]),
            "sdnn_set_weights": (i, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
            "sdnn_get_weights": (i, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
            "sdnn_classify": (i, [vp, vp, vp, vp, vp]),
            "sdnn_indicator": (i, [vp, vp, vp, vp, vp]),
            "sdnn_windows": (i, [vp, vp, vp, vp, vp]),
            "av_assemble": (i, [vp, vp, vp, vp, vp]),
            "sdnn_train_step": (i, [vp, vp, vp, i, ctypes.c_float, vp, vp]),
            "sdnn_gradient": (i, [vp, vp, vp, i, vp, vp, vp]),
            "sdnn_gradient_noalloc": (i, [vp, vp, vp, i, vp, vp, vp]),
            "fcs_step": (i, [vp, vp, d, vp, i, vp]),
            "fcs_filter": (i, [vp, vp, vp]),
            "fcs_smear_initial": (i, [vp, vp, vp, vp]),
            "fcs_step_graph": (i, [vp, vp, d, vp, i, vp]),
            "fcs_status": (i, [vp, ctypes.POINTER(ctypes.c_int)]),
            "fcs_strerror": (ctypes.c_char_p, [i]),
            "fcs_alu_probe": (i, [i, i, i, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(fn, rc):
    if rc != 0:
        raise FcsError(fn, rc)


def build_table(d, C):
    """FP64 continuation table A_R (C x d) from the library's host builder."""
    out = np.zeros((C, d), dtype=np.float64)
    _check("fcs_build_table", lib().fcs_build_table(d, C, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def gradient_noalloc(w, x, labels, grad, loss=None, stream=None):
    """Classifier gradient through sdnn_gradient_noalloc: no context and no
    device allocation inside the library (for callers that cannot allocate).
    w: device float weights (1732); x: device float windows (batch x 16);
    labels: device int8 (batch); grad: device float (1732)."""
    _check("sdnn_gradient_noalloc", lib().sdnn_gradient_noalloc(_ptr(w), _ptr(x), _ptr(labels), int(x.shape[0]),
                                                                _ptr(loss), _ptr(grad), _stream(stream)))


def alu_probe(dtype, blocks, iters, out, stream=None):
    """Launch the library's FMA-rate probe (blocks x 256 x iters x 64 flops);
    out: device tensor of at least `blocks` elements of the dtype."""
    _check("fcs_alu_probe", lib().fcs_alu_probe(int(dtype), int(blocks), int(iters), _ptr(out), _stream(stream)))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Context:
    """An fcs_ctx for one patch layout (an ``inputs.Instance``) and its options."""

    def __init__(self, inst, d=5, C=25, dtype=F32, instances=1, cfl=0.5, n_f=5, c_mu=1.0, av_radius=4,
                 c_policy=0, train_batch_max=4096, autotune=0, filter_step=0, filter_p=None, filter_alpha=None,
                 op_form=0):
        import torch  # device memory and streams
        self.torch = torch
        L = lib()
        self.inst = inst
        self.dtype = dtype
        self.tdtype = torch.float64 if dtype == F64 else torch.float32
        self.npdtype = np.float64 if dtype == F64 else np.float32
        opt = Options()
        L.fcs_default_options(ctypes.byref(opt))
        opt.gamma, opt.cfl, opt.n_f, opt.dtype, opt.instances = inst.gamma, cfl, n_f, dtype, instances
        for k in range(4):
            opt.inflow[k] = inst.inflow[k]
        opt.p_out, opt.c_mu, opt.av_radius, opt.c_policy = inst.p_out, c_mu, av_radius, c_policy
        opt.train_batch_max = train_batch_max
        opt.autotune = autotune
        opt.filter_step = filter_step
        opt.op_form = op_form
        if filter_p is not None:
            opt.filter_p = filter_p
        if filter_alpha is not None:
            opt.filter_alpha = filter_alpha
        descs = (PatchDesc * len(inst.patches))()
        self._keep = []
        for k, p in enumerate(inst.patches):
            descs[k].n1, descs[k].n2 = p.n1, p.n2
            if getattr(p, "is_l", False):
                descs[k].lcut[0], descs[k].lcut[1] = int(p.lcut[0]), int(p.lcut[1])
            if getattr(p, "inflow", None) is not None:
                infl = np.ascontiguousarray(p.inflow, dtype=np.float64)
                self._keep.append(infl)
                descs[k].inflow = infl.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            for s in range(4):
                descs[k].bc[s] = int(p.bc[s])
            if p.cartesian:
                descs[k].cartesian = 1
                for s in range(4):
                    descs[k].box[s] = float(p.box[s])
            else:
                x = np.ascontiguousarray(p.x, dtype=np.float64)
                y = np.ascontiguousarray(p.y, dtype=np.float64)
                self._keep += [x, y]
                descs[k].cartesian = 0
                descs[k].x = x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                descs[k].y = y.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _check("fc_setup", L.fc_setup(ctypes.byref(h), d, C, descs, len(inst.patches), ctypes.byref(opt)))
        self.h = h
        lay = Layout()
        _check("fcs_get_layout", L.fcs_get_layout(h, ctypes.byref(lay)))
        self.instances = lay.instances
        self.npatch = lay.npatch
        self.state_elems = lay.state_elems
        self.scalar_elems = lay.scalar_elems
        self.windows = lay.windows
        self.state_off = [lay.state_off[k] for k in range(self.npatch)]
        self.scalar_off = [lay.scalar_off[k] for k in range(self.npatch)]
        self.window_off = [lay.window_off[k] for k in range(self.npatch)]
        self.tile_width = lay.tile_width
        self.launches = {"stage": lay.launches_stage, "stage_visc": lay.launches_stage_visc,
                         "exchange": lay.launches_exchange, "av": lay.launches_av}
        self.dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else None

    def close(self):
        if getattr(self, "h", None):
            lib().fc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ buffers
    def new_state(self):
        return self.torch.zeros(self.instances * self.state_elems, dtype=self.tdtype, device=self.dev)

    def new_scalar(self, dtype=None):
        return self.torch.zeros(self.instances * self.scalar_elems, dtype=dtype or self.tdtype, device=self.dev)

    def pack_state(self, states):
        """states[instance][patch] -> (4, n2, n1) arrays; returns a flat host array."""
        out = np.zeros(self.instances * self.state_elems, dtype=self.npdtype)
        for k in range(self.instances):
            st = states[k] if isinstance(states[0], (list, tuple)) else states
            for p, e in enumerate(st):
                o = k * self.state_elems + self.state_off[p]
                out[o:o + e.size] = np.asarray(e, dtype=self.npdtype).ravel()
        return out

    def unpack_state(self, flat, instance=0):
        flat = flat.detach().cpu().numpy() if hasattr(flat, "detach") else np.asarray(flat)
        res = []
        for p, pt in enumerate(self.inst.patches):
            o = instance * self.state_elems + self.state_off[p]
            res.append(flat[o:o + 4 * pt.n1 * pt.n2].reshape(4, pt.n2, pt.n1).astype(np.float64))
        return res

    def pack_scalar(self, fields, dtype=None):
        out = np.zeros(self.instances * self.scalar_elems, dtype=dtype or self.npdtype)
        for k in range(self.instances):
            fl = fields[k] if isinstance(fields[0], (list, tuple)) else fields
            for p, f in enumerate(fl):
                o = k * self.scalar_elems + self.scalar_off[p]
                out[o:o + f.size] = np.asarray(f).ravel()
        return out

    def unpack_scalar(self, flat, instance=0):
        flat = flat.detach().cpu().numpy() if hasattr(flat, "detach") else np.asarray(flat)
        res = []
        for p, pt in enumerate(self.inst.patches):
            o = instance * self.scalar_elems + self.scalar_off[p]
            res.append(flat[o:o + pt.n1 * pt.n2].reshape(pt.n2, pt.n1))
        return res

    def to_device(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a)).to(self.dev)

    # ------------------------------------------------------------ entry points
    def fc_derivative(self, x, out, direction, order=1, stream=None):
        _check("fc_derivative", lib().fc_derivative(self.h, _ptr(x), _ptr(out), direction, order, _stream(stream)))

    def euler_rhs(self, e, rhs, mu=None, stream=None):
        _check("euler_rhs", lib().euler_rhs(self.h, _ptr(e), _ptr(mu), _ptr(rhs), _stream(stream)))

    def rk_stage(self, stage, dt, e_n, e_s, acc, out, mu=None, dt_dev=None, stream=None):
        _check("rk_stage", lib().rk_stage(self.h, stage, float(dt), _ptr(dt_dev), _ptr(e_n), _ptr(e_s), _ptr(acc),
                                          _ptr(out), _ptr(mu), _stream(stream)))

    def patch_exchange(self, field, nfields=4, stream=None):
        _check("patch_exchange", lib().patch_exchange(self.h, _ptr(field), nfields, _stream(stream)))

    def time_step(self, e, dt_dev, mu=None, stream=None):
        _check("fcs_time_step", lib().fcs_time_step(self.h, _ptr(e), _ptr(mu), _ptr(dt_dev), _stream(stream)))

    def conservation_sums(self, e, sums, stream=None):
        _check("fcs_conservation_sums", lib().fcs_conservation_sums(self.h, _ptr(e), _ptr(sums), _stream(stream)))

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check("sdnn_set_weights", lib().sdnn_set_weights(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                          w.size))

    def get_weights(self):
        w = np.zeros(N_PARAMS, dtype=np.float32)
        _check("sdnn_get_weights", lib().sdnn_get_weights(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                          w.size))
        return w

    def classify(self, e, tau, logits=None, stream=None):
        _check("sdnn_classify", lib().sdnn_classify(self.h, _ptr(e), _ptr(tau), _ptr(logits), _stream(stream)))

    def windows_raw(self, e, x, flat=None, stream=None):
        """Raw proxy windows (instances x windows x 16 float) and flat flags."""
        _check("sdnn_windows", lib().sdnn_windows(self.h, _ptr(e), _ptr(x), _ptr(flat), _stream(stream)))

    def indicator(self, e, tau, s=None, stream=None):
        _check("sdnn_indicator", lib().sdnn_indicator(self.h, _ptr(e), _ptr(tau), _ptr(s), _stream(stream)))

    def av_assemble(self, e, tau, mu, stream=None):
        _check("av_assemble", lib().av_assemble(self.h, _ptr(e), _ptr(tau), _ptr(mu), _stream(stream)))

    def train_step(self, x, labels, lr, loss=None, stream=None):
        _check("sdnn_train_step", lib().sdnn_train_step(self.h, _ptr(x), _ptr(labels), int(x.shape[0]),
                                                        ctypes.c_float(lr), _ptr(loss), _stream(stream)))

    def gradient(self, x, labels, grad, loss=None, stream=None):
        _check("sdnn_gradient", lib().sdnn_gradient(self.h, _ptr(x), _ptr(labels), int(x.shape[0]), _ptr(loss),
                                                    _ptr(grad), _stream(stream)))

    def line_c(self, N):
        """Continuation length the context uses on lines of N points."""
        return int(lib().fcs_line_c(self.h, int(N)))

    def filter(self, e, stream=None):
        _check("fcs_filter", lib().fcs_filter(self.h, _ptr(e), _stream(stream)))

    def smear_initial(self, e, tau, stream=None):
        _check("fcs_smear_initial", lib().fcs_smear_initial(self.h, _ptr(e), _ptr(tau), _stream(stream)))

    def step(self, e, dt=0.0, dt_dev=None, use_av=False, stream=None):
        _check("fcs_step", lib().fcs_step(self.h, _ptr(e), float(dt), _ptr(dt_dev), int(use_av), _stream(stream)))

    def step_graph(self, e, dt=0.0, dt_dev=None, use_av=False, stream=None):
        _check("fcs_step_graph", lib().fcs_step_graph(self.h, _ptr(e), float(dt), _ptr(dt_dev), int(use_av),
                                                      _stream(stream)))

    def status(self):
        f = ctypes.c_int(0)
        rc = lib().fcs_status(self.h, ctypes.byref(f))
        return rc, f.value
