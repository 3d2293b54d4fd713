"""ctypes binding of the FLNR guide network in libflr.so (include/flr.h, flnr_*).

Argument marshalling only: the forward and backward passes, the loss and the optimiser
run in the library's kernels.  FLNR (Sec. 3.3) turns the guides and noisy radiance into
enhanced guides for FLR; training through FLR's adjoint is in flnr_train.py.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import flr as _flr

# (name, cin, cout, kernel) in the library's order; the flat parameter array holds each
# layer's weights [cout][cin][k][k] and then its biases [cout].  The head o1 has 8 outputs,
# or 16 for the two guide sets of Sec. 3.3 (layers(16)).
def layers(outputs=8):
    return [("in0", 11, 16, 3), ("in1", 16, 16, 1), ("e1a", 16, 32, 3), ("e1b", 32, 32, 3),
            ("e2a", 32, 64, 3), ("e2b", 64, 64, 3), ("d1a", 96, 32, 3), ("d1b", 32, 32, 3),
            ("d0a", 48, 16, 3), ("d0b", 16, 16, 3), ("o0", 16, 16, 3), ("o1", 16, outputs, 1)]


LAYERS = layers(8)
_bound = False


def _lib():
    global _bound
    lib = _flr.load_library()
    if not _bound:
        vp, ip = ctypes.c_void_p, ctypes.c_int
        lib.flnr_param_count.restype = ctypes.c_size_t
        lib.flnr_param_count.argtypes = [ip]
        lib.flnr_create.argtypes = [ip, ip, ctypes.POINTER(ctypes.c_void_p)]
        lib.flnr_destroy.argtypes = [vp]
        lib.flnr_set_weights.argtypes = [vp, vp, ctypes.c_size_t]
        lib.flnr_get_weights.argtypes = [vp, vp, ctypes.c_size_t]
        lib.flnr_get_grads.argtypes = [vp, vp, ctypes.c_size_t]
        lib.flnr_get_state.argtypes = [vp, vp, ctypes.c_size_t]
        lib.flnr_set_state.argtypes = [vp, vp, ctypes.c_size_t]
        lib.flnr_guide_forward.argtypes = [vp, vp, vp, ip, ip, ip, vp]
        lib.flnr_guide_backward.argtypes = [vp, vp, vp, vp]
        lib.flnr_zero_grads.argtypes = [vp, vp]
        lib.flnr_adam_step.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ip, vp]
        lib.flnr_l1_loss.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp]
        lib.flnr_smape_loss.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, ctypes.c_float, vp]
        lib.flnr_layer.argtypes = [vp, ip, ip, vp, vp, vp, vp, ip, ip, ip, vp]
        lib.flnr_status.argtypes = [vp]
        for name in ("flnr_create", "flnr_destroy", "flnr_set_weights", "flnr_get_weights", "flnr_get_grads",
                     "flnr_get_state", "flnr_set_state", "flnr_guide_forward", "flnr_guide_backward",
                     "flnr_zero_grads", "flnr_adam_step",
                     "flnr_l1_loss", "flnr_smape_loss", "flnr_layer", "flnr_status"):
            getattr(lib, name).restype = ctypes.c_int
        _bound = True
    return lib


def init_weights(seed=0, outputs=8):
    """Seeded initial parameters (dict name.w / name.b, float32): He-uniform weights, zero
    biases, and the output projection o1 (`outputs` channels) at a tenth of its He bound, so
    that the enhanced guides start near 0.5 with small contrast and the sigmoid starts
    unsaturated.  With 16 outputs the map rows of o1 start as a copy of the model rows."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, cin, cout, k in layers(outputs):
        bound = np.sqrt(6.0 / (cin * k * k)) * (0.1 if name == "o1" else 1.0)
        params[name + ".w"] = rng.uniform(-bound, bound, size=(cout, cin, k, k)).astype(np.float32)
        params[name + ".b"] = np.zeros(cout, np.float32)
    if outputs == 16:  # the map set starts as a copy of the model set
        params["o1.w"][8:] = params["o1.w"][:8]
    return params


def flatten(params):
    """dict name.w / name.b -> flat float32 array in the library's order."""
    return np.concatenate([np.concatenate([np.asarray(params[n + ".w"], np.float32).ravel(),
                                           np.asarray(params[n + ".b"], np.float32).ravel()])
                           for n, _, _, _ in LAYERS])


def unflatten(flat, outputs=8):
    out, o = {}, 0
    for n, ci, co, k in layers(outputs):
        out[n + ".w"] = flat[o:o + co * ci * k * k].reshape(co, ci, k, k)
        o += co * ci * k * k
        out[n + ".b"] = flat[o:o + co]
        o += co
    return out


def _stream(t):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


class FLNR:
    """The guide network: forward, backward (accumulating), Adam, on CUDA tensors."""

    def __init__(self, max_pixels, weights, outputs=None):
        """outputs: 8 (one guide set) or 16 (model and map sets, Sec. 3.3); by default the
        size of the weights' output layer."""
        lib = _lib()
        if outputs is None:
            outputs = int(np.asarray(weights["o1.b"]).size) if isinstance(weights, dict) else 8
        self.outputs = int(outputs)
        h = ctypes.c_void_p()
        _flr._check(lib.flnr_create(int(max_pixels), self.outputs, ctypes.byref(h)), "flnr_create")
        self._h = h
        self.count = int(lib.flnr_param_count(self.outputs))
        self.set_weights(weights)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().flnr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, weights):
        flat = flatten(weights) if isinstance(weights, dict) else np.ascontiguousarray(weights, np.float32)
        if flat.size != self.count:
            raise ValueError(f"expected {self.count} parameters, got {flat.size}")
        _flr._check(_lib().flnr_set_weights(self._h, flat.ctypes.data, flat.size), "flnr_set_weights")

    def get_weights(self):
        flat = np.empty(self.count, np.float32)
        _flr._check(_lib().flnr_get_weights(self._h, flat.ctypes.data, flat.size), "flnr_get_weights")
        return flat

    def get_state(self):
        """Master weights, Adam first and second moments: float32 [3 * count] (host)."""
        flat = np.empty(3 * self.count, np.float32)
        _flr._check(_lib().flnr_get_state(self._h, flat.ctypes.data, flat.size), "flnr_get_state")
        return flat

    def set_state(self, state):
        """Restores what get_state returned (weights and Adam moments, exactly)."""
        flat = np.ascontiguousarray(state, np.float32)
        if flat.size != 3 * self.count:
            raise ValueError(f"expected {3 * self.count} floats, got {flat.size}")
        _flr._check(_lib().flnr_set_state(self._h, flat.ctypes.data, flat.size), "flnr_set_state")

    def grads(self):
        flat = np.empty(self.count, np.float32)
        _flr._check(_lib().flnr_get_grads(self._h, flat.ctypes.data, flat.size), "flnr_get_grads")
        return flat

    def forward(self, x, out=None):
        """x [N,11,H,W] CUDA float32 -> enhanced guides [N,outputs,H,W] float32."""
        import torch
        N, C, H, W = (int(v) for v in x.shape)
        if C != 11 or not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
            raise TypeError("x must be a contiguous CUDA float32 [N, 11, H, W] tensor")
        if out is None:
            out = torch.empty((N, self.outputs, H, W), dtype=torch.float32, device=x.device)
        _flr._check(_lib().flnr_guide_forward(self._h, x.data_ptr(), out.data_ptr(), N, H, W, _stream(x)),
                    "flnr_guide_forward")
        return out

    def backward(self, grad_out, grad_in=None):
        """Accumulate parameter gradients for dL/d(enhanced guides) = grad_out [N,outputs,H,W];
        grad_in (optional CUDA float32 [N,11,H,W]) receives dL/d(input)."""
        gi = None if grad_in is None else ctypes.c_void_p(grad_in.data_ptr())
        _flr._check(_lib().flnr_guide_backward(self._h, grad_out.contiguous().data_ptr(), gi, _stream(grad_out)),
                    "flnr_guide_backward")
        return grad_in

    OP_FORWARD, OP_DGRAD, OP_WGRAD = 0, 1, 2

    def status(self):
        """Waits for the device; raises if a tensor-core kernel's bounded wait ran out."""
        _flr._check(_lib().flnr_status(self._h), "flnr_status")

    def layer(self, layer, op, a, b=None, mask=None, out=None, size=None):
        """One layer's kernels by themselves (flnr_layer): a, b, mask, out are CUDA bfloat16
        NHWC tensors with padded channels (out float32 planar for layer 11's forward).  The
        layer's input size [N, H, W] comes from `a`, or from `size` when `a` is not at that
        size (the half-resolution input of a decoder layer, or the gradient dz of a stride-2
        layer)."""
        N, H, W = (int(v) for v in (size if size is not None else a.shape[:3]))
        ptr = (lambda t: None if t is None else ctypes.c_void_p(t.data_ptr()))
        _flr._check(_lib().flnr_layer(self._h, int(layer), int(op), ptr(a), ptr(b), ptr(mask), ptr(out),
                                      N, H, W, _stream(a)), "flnr_layer")
        return out

    def zero_grads(self, stream_of):
        _flr._check(_lib().flnr_zero_grads(self._h, _stream(stream_of)), "flnr_zero_grads")

    def adam_step(self, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream_of=None):
        import torch
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream) if stream_of is None else _stream(stream_of)
        _flr._check(_lib().flnr_adam_step(self._h, lr, beta1, beta2, eps, int(step), st), "flnr_adam_step")


def l1_loss(pred, ref):
    """Mean absolute error and its gradient, computed by the library's kernel."""
    import torch
    grad = torch.empty_like(pred)
    loss = torch.empty(1, dtype=torch.float32, device=pred.device)
    _flr._check(_lib().flnr_l1_loss(pred.data_ptr(), ref.data_ptr(), grad.data_ptr(), loss.data_ptr(),
                                    pred.numel(), _stream(pred)), "flnr_l1_loss")
    return loss, grad


def smape_loss(pred, ref, eps=1e-2):
    """SMAPE mean |p - r| / (|p| + |r| + eps) and its gradient (Sec. 3.3's training loss),
    computed by the library's kernel."""
    import torch
    grad = torch.empty_like(pred)
    loss = torch.empty(1, dtype=torch.float32, device=pred.device)
    _flr._check(_lib().flnr_smape_loss(pred.data_ptr(), ref.data_ptr(), grad.data_ptr(), loss.data_ptr(),
                                       pred.numel(), float(eps), _stream(pred)), "flnr_smape_loss")
    return loss, grad
