"""Python layer over the C ABI: handles, torch-owned device buffers, and a
``torch.autograd.Function`` for the FastVPINNs loss.

PyTorch provides device memory and the CUDA stream; every computation of the
loss path (G precompute, MLP forward + tangents, contraction, adjoint, MLP
reverse, Adam) runs in the CUDA library through ``_native``.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _native as N

PRECISIONS = {"fp64": N.FV_FP64, "fp32": N.FV_FP32, "tf32": N.FV_TF32, "bf16": N.FV_BF16, "fp16": N.FV_FP16}
NORMS = {"test": N.FV_NORM_TEST, "elem": N.FV_NORM_ELEM}


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _host(a, dtype=np.float64) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def param_dtype(precision) -> torch.dtype:
    return torch.float64 if _prec(precision) == N.FV_FP64 else torch.float32


class Context:
    """A library context bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = C.c_void_p()
        N.call("fv_ctx_create", C.byref(h), device, C.c_void_p(self.stream.cuda_stream))
        self.h = h

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        N.call("fv_ctx_set_stream", self.h, C.c_void_p(stream.cuda_stream))

    def enable_timing(self, on: bool = True):
        N.call("fv_ctx_enable_timing", self.h, int(on))

    def set_activation_stash(self, on: bool = True):
        """Tensor-core reverse sweep: read the forward's stored hidden
        activations (on, the default) or recompute them (off); bitwise equal."""
        N.call("fv_ctx_set_activation_stash", self.h, int(on))

    def kernel_times(self) -> dict:
        ms = (C.c_double * 32)()
        ln = (C.c_int64 * 32)()
        n = C.c_int()
        N.call("fv_ctx_kernel_times", self.h, 32, ms, ln, C.byref(n))
        out = {}
        for i in range(min(n.value, 32)):
            if ln[i]:
                out[N.lib().fv_kernel_name(i).decode()] = (ms[i], int(ln[i]))
        return out

    def reset_kernel_times(self):
        N.call("fv_ctx_reset_kernel_times", self.h)

    def close(self):
        if getattr(self, "h", None):
            N.lib().fv_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """Stacked premultiplier tensors of one quad mesh (fv_build_mesh_tensors)."""

    def __init__(self, ctx: Context, vertices, cells, quad_order: int, test_order: int, storage="fp32",
                 with_mass_term: bool = False):
        self.ctx = ctx
        v = _host(vertices).reshape(-1, 2)
        c = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 4)
        h = C.c_void_p()
        N.call("fv_build_mesh_tensors", ctx.h, v.shape[0], v.ctypes.data, c.shape[0], c.ctypes.data,
               quad_order, test_order, _prec(storage), int(with_mass_term), C.byref(h))
        self.h = h
        info = (C.c_int64 * 8)()
        N.call("fv_mesh_info", h, info)
        self.n_elements, self.Nq, self.Nt, self.n_points, self.n_comp = (int(info[i]) for i in range(5))
        self.g_bytes_stored, self.g_bytes = int(info[5]), int(info[6])
        self.storage = int(info[7])
        self.Q, self.T = quad_order, test_order

    def quad_points(self) -> np.ndarray:
        out = np.zeros((self.n_points, 2))
        N.call("fv_mesh_quad_points", self.h, out.ctypes.data)
        return out

    def g_tensor(self) -> np.ndarray:
        out = np.zeros((self.n_elements, self.n_comp, self.Nt, self.Nq))
        N.call("fv_mesh_copy_g", self.h, out.ctypes.data)
        return out

    def set_g_mode(self, mode: str = "stored"):
        """'stored' streams the stored G tensor; 'matrix_free' rebuilds it in
        the contraction from the element vertices; 'regular' (axis-aligned
        rectangles only) runs Alg. 2's reference-matrix GEMMs on the tensor
        cores (fv_mesh_set_g_mode)."""
        m = {"stored": N.FV_G_STORED, "matrix_free": N.FV_G_MATRIX_FREE, "regular": N.FV_G_REGULAR}[mode]
        N.call("fv_mesh_set_g_mode", self.h, m)
        self.g_mode = mode

    def autotune(self, precision="fp32") -> tuple:
        """Time the contraction's launch plans for this mesh at `precision`
        and keep the fastest (fv_autotune).  Returns the median milliseconds
        of the best two-stage and the best one-stage candidate."""
        ms = (C.c_double * 2)()
        N.call("fv_autotune", self.ctx.h, self.h, _prec(precision), ms)
        return ms[0], ms[1]

    def close(self):
        if getattr(self, "h", None):
            N.lib().fv_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Forcing:
    def __init__(self, mesh: Mesh, f_at_quad):
        self.mesh = mesh
        f = _host(f_at_quad).reshape(-1)
        if f.size != mesh.n_points:
            raise ValueError("f must have one value per quadrature point")
        h = C.c_void_p()
        N.call("fv_assemble_forcing", mesh.h, f.ctypes.data, C.byref(h))
        self.h = h

    def matrix(self) -> np.ndarray:
        out = np.zeros((self.mesh.n_elements, self.mesh.Nt))
        N.call("fv_forcing_copy", self.h, out.ctypes.data)
        return out

    def close(self):
        if getattr(self, "h", None):
            N.lib().fv_forcing_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BC:
    def __init__(self, ctx: Context, bd_xy=None, bd_g=None, tau: float = 1.0, s_xy=None, s_u=None,
                 gamma: float = 1.0):
        self.ctx = ctx
        bxy = _host(bd_xy if bd_xy is not None else np.zeros((0, 2))).reshape(-1, 2)
        bg = _host(bd_g if bd_g is not None else np.zeros(0)).reshape(-1)
        sxy = _host(s_xy if s_xy is not None else np.zeros((0, 2))).reshape(-1, 2)
        su = _host(s_u if s_u is not None else np.zeros(0)).reshape(-1)
        self.n_bd, self.n_s = bxy.shape[0], sxy.shape[0]
        h = C.c_void_p()
        N.call("fv_bc_create", ctx.h, self.n_bd, bxy.ctypes.data if self.n_bd else None,
               bg.ctypes.data if self.n_bd else None, float(tau), self.n_s, sxy.ctypes.data if self.n_s else None,
               su.ctypes.data if self.n_s else None, float(gamma), C.byref(h))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            N.lib().fv_bc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Network:
    def __init__(self, widths: Sequence[int]):
        self.widths = list(int(w) for w in widths)
        self._w = (C.c_int * len(self.widths))(*self.widths)
        self.desc = N.fv_mlp_desc(len(self.widths) - 1, self._w)
        self.n_params = sum(self.widths[i + 1] * (self.widths[i] + 1) for i in range(len(self.widths) - 1))


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


class Problem:
    """Everything one loss evaluation needs, bound to a context."""

    def __init__(self, ctx: Context, mesh: Mesh, forcing: Forcing, bc: Optional[BC], widths, precision="fp32",
                 eps: float = 1.0, b=(0.0, 0.0), norm="test"):
        self.ctx, self.mesh, self.forcing, self.bc = ctx, mesh, forcing, bc
        self.net = Network(widths)
        self.precision = _prec(precision)
        self.eps, self.b = float(eps), (float(b[0]), float(b[1]))
        self.norm = NORMS[norm] if isinstance(norm, str) else int(norm)
        dev = torch.device("cuda", ctx.device)
        self.out = torch.zeros(5, dtype=torch.float64, device=dev)
        self.dtype = param_dtype(self.precision)

    def opts(self, eps_dev: Optional[torch.Tensor] = None) -> N.fv_eval_opts:
        return N.fv_eval_opts(self.precision, self.eps, _ptr(eps_dev), self.b[0], self.b[1], self.norm)

    def _check_params(self, params: torch.Tensor):
        if not params.is_cuda or params.dtype != self.dtype or not params.is_contiguous() \
                or params.numel() != self.net.n_params:
            raise ValueError("params must be a contiguous CUDA %s tensor of %d values"
                             % (self.dtype, self.net.n_params))

    def _check_outputs(self, params: torch.Tensor, grad: Optional[torch.Tensor], out: Optional[torch.Tensor],
                       n_out: int):
        """The library writes n_params values to grad and n_out doubles to out
        without bounds: a short, strided, wrongly typed or host tensor would be
        an out-of-bounds device write, so it is refused here."""
        if grad is not None and (not grad.is_cuda or grad.device != params.device or grad.dtype != self.dtype
                                 or not grad.is_contiguous() or grad.numel() != self.net.n_params):
            raise ValueError("grad must be a contiguous %s tensor of %d values on %s"
                             % (self.dtype, self.net.n_params, params.device))
        if out is not None and (not out.is_cuda or out.device != params.device or out.dtype != torch.float64
                                or not out.is_contiguous() or out.numel() < n_out):
            raise ValueError("out must be a contiguous float64 tensor of at least %d values on %s"
                             % (n_out, params.device))

    def loss(self, params: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        self._check_params(params)
        self._check_outputs(params, None, out, 4)
        out = self.out if out is None else out
        o = self.opts()
        N.call("fv_loss", self.ctx.h, self.mesh.h, self.forcing.h, self.bc.h if self.bc else None,
               C.byref(self.net.desc), _ptr(params), C.byref(o), _ptr(out))
        return out[:4]

    def loss_grad(self, params: torch.Tensor, grad: Optional[torch.Tensor] = None,
                  out: Optional[torch.Tensor] = None):
        """Returns (out, grad): out = (L, Lv, Lb, Ls, dL/deps) on the device."""
        self._check_params(params)
        self._check_outputs(params, grad, out, 5)
        grad = torch.empty_like(params) if grad is None else grad
        out = self.out if out is None else out
        o = self.opts()
        N.call("fv_loss_grad", self.ctx.h, self.mesh.h, self.forcing.h, self.bc.h if self.bc else None,
               C.byref(self.net.desc), _ptr(params), C.byref(o), _ptr(grad), _ptr(out))
        return out, grad

    def loss_grad_noalloc(self, params: torch.Tensor, grad: torch.Tensor, out: torch.Tensor):
        """fv_loss_grad_noalloc: as loss_grad, with every temporary in the
        library's fixed scratch area (for callers that cannot allocate device
        memory); grad and out must be supplied."""
        self._check_params(params)
        if grad is None or out is None:
            raise ValueError("loss_grad_noalloc needs caller-supplied grad and out tensors")
        self._check_outputs(params, grad, out, 5)
        o = self.opts()
        N.call("fv_loss_grad_noalloc", self.ctx.h, self.mesh.h, self.forcing.h, self.bc.h if self.bc else None,
               C.byref(self.net.desc), _ptr(params), C.byref(o), _ptr(grad), _ptr(out))
        return out, grad

    def intermediates(self, params: torch.Tensor):
        """(out, U [S][P_tot], UB [S][P_tot], R [n_e][T*T]) of one evaluation; S = 3,
        or 4 for a two-output network (eps(x, y) and its seed last)."""
        self._check_params(params)
        P_tot = self.mesh.n_points + (self.bc.n_bd + self.bc.n_s if self.bc else 0)
        U = torch.empty(2 + self.net.widths[-1], P_tot, dtype=self.dtype, device=params.device)
        UB = torch.empty_like(U)
        R = torch.empty(self.mesh.n_elements, self.mesh.Nt, dtype=torch.float64, device=params.device)
        out = torch.zeros(5, dtype=torch.float64, device=params.device)
        o = self.opts()
        N.call("fv_eval_intermediates", self.ctx.h, self.mesh.h, self.forcing.h, self.bc.h if self.bc else None,
               C.byref(self.net.desc), _ptr(params), C.byref(o), _ptr(U), _ptr(UB), _ptr(R), _ptr(out))
        return out, U, UB, R

    def inverse_step(self, params: torch.Tensor, eps_dev: torch.Tensor, adam: Optional["Adam"], lr: float,
                     grad: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None):
        self._check_params(params)
        self._check_outputs(params, grad, out, 5)
        grad = torch.empty_like(params) if grad is None else grad
        out = self.out if out is None else out
        o = self.opts(eps_dev)
        N.call("fv_inverse_step", self.ctx.h, self.mesh.h, self.forcing.h, self.bc.h if self.bc else None,
               C.byref(self.net.desc), _ptr(params), _ptr(eps_dev), C.byref(o), adam.h if adam else None,
               float(lr), _ptr(grad), _ptr(out))
        return out, grad


class StepGraph:
    """n_steps training steps (loss + gradient + Adam) captured into one CUDA
    graph (fv_step_graph_create); launch() replays them with one host call.
    The tensors given at creation are updated in place on every launch."""

    def __init__(self, problem: "Problem", params: torch.Tensor, eps_dev: torch.Tensor, adam: Optional["Adam"],
                 lr: float, n_steps: int = 1, grad: Optional[torch.Tensor] = None,
                 out: Optional[torch.Tensor] = None):
        problem._check_params(params)
        self.problem, self.params, self.eps_dev, self.adam = problem, params, eps_dev, adam
        self.grad = torch.empty_like(params) if grad is None else grad
        self.out = torch.zeros(5, dtype=torch.float64, device=params.device) if out is None else out
        self.n_steps = n_steps
        self._opts = problem.opts(eps_dev)
        h = C.c_void_p()
        N.call("fv_step_graph_create", problem.ctx.h, problem.mesh.h, problem.forcing.h,
               problem.bc.h if problem.bc else None, C.byref(problem.net.desc), _ptr(params), _ptr(eps_dev),
               C.byref(self._opts), adam.h if adam else None, float(lr), _ptr(self.grad), _ptr(self.out),
               int(n_steps), C.byref(h))
        self.h = h

    def launch(self):
        N.call("fv_graph_launch", self.h)
        return self.out, self.grad

    def close(self):
        if getattr(self, "h", None):
            N.call("fv_graph_destroy", self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adam:
    def __init__(self, ctx: Context, n_params: int, precision="fp32", beta1=0.9, beta2=0.999, eps=1e-8,
                 with_eps: bool = True):
        h = C.c_void_p()
        N.call("fv_adam_create", ctx.h, n_params, _prec(precision), beta1, beta2, eps, int(with_eps), C.byref(h))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            N.lib().fv_adam_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_eval(ctx: Context, widths, params: torch.Tensor, xy: torch.Tensor, precision=None) -> torch.Tensor:
    """(u, u_x, u_y[, eps]) of the network at device points xy [n][2] (FP64)."""
    net = Network(widths)
    prec = _prec(precision) if precision is not None else (N.FV_FP64 if params.dtype == torch.float64 else N.FV_FP32)
    xy = xy.to(torch.float64).contiguous()
    out = torch.empty(2 + int(widths[-1]), xy.shape[0], dtype=params.dtype, device=params.device)
    N.call("fv_mlp_eval", ctx.h, C.byref(net.desc), _ptr(params), prec, xy.shape[0], _ptr(xy), _ptr(out))
    return out


class FastVPINNLoss(torch.autograd.Function):
    """loss = FastVPINNLoss.apply(params, problem): the FastVPINNs loss with its
    gradient from the library's fused forward + adjoint pass."""

    @staticmethod
    def forward(fctx, params: torch.Tensor, problem: Problem):
        out, grad = problem.loss_grad(params.detach().contiguous())
        fctx.save_for_backward(grad)
        return out[0].to(params.dtype).clone()

    @staticmethod
    def backward(fctx, g):
        (grad,) = fctx.saved_tensors
        return g * grad, None


class Batch:
    """Loss + gradient of many independent problems in one call (fv_batch_*)."""

    def __init__(self, ctx: Context, problems: Sequence[Problem], params: Sequence[torch.Tensor], n_streams: int = 0):
        self.ctx, self.problems, self.params = ctx, list(problems), list(params)
        p0 = self.problems[0]
        self.grads = [torch.empty_like(p) for p in self.params]
        self.outs = [torch.zeros(5, dtype=torch.float64, device=p.device) for p in self.params]
        arr = (N.fv_instance * len(self.problems))()
        for i, (pb, p) in enumerate(zip(self.problems, self.params)):
            arr[i] = N.fv_instance(pb.mesh.h.value, pb.forcing.h.value, pb.bc.h.value if pb.bc else None,
                                   p.data_ptr(), self.grads[i].data_ptr(), self.outs[i].data_ptr())
        self._arr = arr
        o = p0.opts()
        h = C.c_void_p()
        N.call("fv_batch_plan", ctx.h, len(self.problems), arr, C.byref(p0.net.desc), C.byref(o), int(n_streams),
               C.byref(h))
        self.h = h

    def info(self):
        n = C.c_int()
        t = (C.c_double * 4)()
        N.call("fv_batch_info", self.h, C.byref(n), t)
        return n.value, list(t)

    def run(self):
        N.call("fv_batch_loss_grad", self.h)
        return self.outs, self.grads

    def close(self):
        if getattr(self, "h", None):
            N.lib().fv_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def problem_from_inputs(ctx: Context, prob, precision="fp32", storage=None, norm="test", with_bc=True,
                        mesh: Optional[Mesh] = None, g_mode: Optional[str] = None) -> Problem:
    """Build the library handles for a problem description with fields mesh
    (vertices, cells), quad_order, test_order, widths, f(x, y), bd_xy, bd_g,
    tau, sensor_xy, sensor_u, gamma, eps, b (duck-typed).  g_mode
    ('stored' / 'matrix_free' / 'regular') sets the mesh's contraction mode."""
    prec = _prec(precision)
    if storage is None:
        storage = "fp64" if prec == N.FV_FP64 else "fp32"
    with_mass = prob.b[0] != 0.0 or prob.b[1] != 0.0
    if mesh is None:
        mesh = Mesh(ctx, prob.mesh.vertices, prob.mesh.cells, prob.quad_order, prob.test_order, storage, with_mass)
    if g_mode is not None:
        mesh.set_g_mode(g_mode)
    X = mesh.quad_points()
    forcing = Forcing(mesh, prob.f(X[:, 0], X[:, 1]))
    bc = None
    if with_bc and (len(prob.bd_xy) or len(prob.sensor_xy)):
        bc = BC(ctx, prob.bd_xy, prob.bd_g, prob.tau, prob.sensor_xy if len(prob.sensor_xy) else None,
                prob.sensor_u if len(prob.sensor_u) else None, prob.gamma)
    return Problem(ctx, mesh, forcing, bc, prob.widths, precision, prob.eps, prob.b, norm)
