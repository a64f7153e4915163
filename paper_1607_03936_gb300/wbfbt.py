"""ctypes binding of libwbfbt.so (include/wbfbt.h): argument marshalling only.

Every numerical step runs inside the CUDA library; this module turns torch
tensors into raw pointers and the current CUDA stream into a cudaStream_t.
Importing it loads the library and raises if it is missing: there is no
fallback.
"""
from __future__ import annotations

import ctypes
import json
import os
from dataclasses import dataclass

import torch

from . import build as _build

F64, F32 = 0, 1
MIXED = 1
ELEM_AUTO, ELEM_POINT, ELEM_ROW = 0, 1, 2   # k = 2 element kernels: by level size, per point, row segments
SCHUR_WBFBT, SCHUR_MASS, SCHUR_MASS_DIAG = 0, 1, 2   # S~: w-BFBT (Eq. wbfbt), lumped M_p(1/mu), diag M_p(1/mu)
BLOCK_A, BLOCK_KL, BLOCK_KR = 0, 1, 2                # blocks for solve_block
WEIGHTS_SQRT_MU, WEIGHTS_GRAD, WEIGHTS_DIAG_A = 0, 1, 2   # C, D: M~_u(sqrt(mu)), M~_u((mu^2+|grad mu|^2)^1/4), diag(A)
OK, ERR_INVALID, ERR_CUDA, ERR_NONFINITE, ERR_BREAKDOWN, ERR_MAXIT, ERR_SETUP = 0, -1, -2, -3, -4, -5, -6
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "non-finite value", -4: "Krylov breakdown",
          -5: "iteration limit reached", -6: "setup failed"}

SYMBOLS = ["wbfbt_default_opts", "wbfbt_sinker_setup", "wbfbt_create", "wbfbt_setup", "wbfbt_apply_A", "wbfbt_apply_B",
           "wbfbt_apply_BT", "wbfbt_apply_K", "wbfbt_apply_Kw", "wbfbt_apply_Ainv", "wbfbt_apply_Kinv",
           "wbfbt_apply_schur_inv", "wbfbt_apply_precond", "wbfbt_solve", "wbfbt_sizes", "wbfbt_device_bytes", "wbfbt_launch_count",
           "wbfbt_destroy", "wbfbt_status_string", "wbfbt_apply_Kw_noalloc",
           "wbfbt_net_num_params", "wbfbt_net_create", "wbfbt_net_set_params", "wbfbt_net_get_params",
           "wbfbt_net_param_count", "wbfbt_net_forward", "wbfbt_net_loss_grad", "wbfbt_net_adam_step",
           "wbfbt_net_save", "wbfbt_net_load", "wbfbt_net_destroy", "wbfbt_attach_net", "wbfbt_learned_sample",
           "wbfbt_learned_stats", "wbfbt_load_learned", "wbfbt_train_learned", "wbfbt_net_conv_layer",
           "wbfbt_solve_block", "wbfbt_set_geometry", "wbfbt_sinker_setup_at", "wbfbt_node_coords"]
NOALLOC_MAX_NODES = 1 << 19


class WbfbtError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status})")
        self.status = status


class Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("a_l", ctypes.c_double), ("a_r", ctypes.c_double), ("restart", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("mg_min_n", ctypes.c_int), ("precision", ctypes.c_int),
                ("schur_sign", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("elem_kernels", ctypes.c_int), ("schur", ctypes.c_int), ("arnoldi_precision", ctypes.c_int),
                ("weights", ctypes.c_int), ("kinv_cycles", ctypes.c_int), ("pmg", ctypes.c_int),
                ("ainv_cycles", ctypes.c_int)]


def library_path() -> str:
    return _build.LIB


def load_library(path: str | None = None) -> ctypes.CDLL:
    path = path or library_path()
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: build it with paper_1607_03936_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.wbfbt_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.wbfbt_default_opts.restype = None
    lib.wbfbt_sinker_setup.argtypes = [ctypes.POINTER(Mesh), i, vp, i, d, d, d, d, vp, vp, vp]
    lib.wbfbt_create.argtypes = [ctypes.POINTER(Mesh), i, vp, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    lib.wbfbt_setup.argtypes = [vp, vp]
    for name in ("wbfbt_apply_A", "wbfbt_apply_B", "wbfbt_apply_BT", "wbfbt_apply_K", "wbfbt_apply_Ainv",
                 "wbfbt_apply_schur_inv", "wbfbt_apply_precond"):
        getattr(lib, name).argtypes = [vp, vp, vp, i]
    lib.wbfbt_apply_Kw.argtypes = [vp, i, vp, vp, i]
    lib.wbfbt_apply_Kinv.argtypes = [vp, i, vp, vp, i]
    lib.wbfbt_solve.argtypes = [vp, vp, vp, vp, d, i, ctypes.POINTER(i), ctypes.POINTER(d)]
    lib.wbfbt_solve_block.argtypes = [vp, i, vp, vp, d, i, ctypes.POINTER(i), ctypes.POINTER(d)]
    lib.wbfbt_set_geometry.argtypes = [vp, vp]
    lib.wbfbt_sinker_setup_at.argtypes = [ctypes.POINTER(Mesh), i, vp, vp, i, d, d, d, d, vp, vp, vp]
    lib.wbfbt_node_coords.argtypes = [ctypes.POINTER(Mesh), i, vp, vp]
    lib.wbfbt_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.wbfbt_device_bytes.argtypes = [vp]
    lib.wbfbt_device_bytes.restype = ctypes.c_longlong
    lib.wbfbt_launch_count.argtypes = []
    lib.wbfbt_launch_count.restype = ctypes.c_longlong
    lib.wbfbt_destroy.argtypes = [vp]
    lib.wbfbt_destroy.restype = None
    lib.wbfbt_apply_Kw_noalloc.argtypes = [ctypes.POINTER(Mesh), i, vp, d, vp, vp, vp]
    lib.wbfbt_net_num_params.argtypes = [i, i]
    lib.wbfbt_net_num_params.restype = ctypes.c_longlong
    lib.wbfbt_net_create.argtypes = [i, i, i, i, vp, ctypes.POINTER(vp)]
    lib.wbfbt_net_set_params.argtypes = [vp, vp]
    lib.wbfbt_net_get_params.argtypes = [vp, vp]
    lib.wbfbt_net_param_count.argtypes = [vp]
    lib.wbfbt_net_param_count.restype = ctypes.c_longlong
    lib.wbfbt_net_forward.argtypes = [vp, vp, i, vp]
    lib.wbfbt_net_loss_grad.argtypes = [vp, vp, vp, i, ctypes.POINTER(d), vp]
    lib.wbfbt_net_adam_step.argtypes = [vp, ctypes.c_float]
    lib.wbfbt_net_save.argtypes = [vp, ctypes.c_char_p]
    lib.wbfbt_net_load.argtypes = [vp, ctypes.c_char_p]
    lib.wbfbt_net_destroy.argtypes = [vp]
    lib.wbfbt_net_destroy.restype = None
    lib.wbfbt_net_conv_layer.argtypes = [vp, i, i, i, vp, vp, vp, vp]
    lib.wbfbt_attach_net.argtypes = [vp, vp, i, d]
    lib.wbfbt_learned_sample.argtypes = [vp, i, vp, vp, vp]
    lib.wbfbt_learned_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.wbfbt_load_learned.argtypes = [vp, ctypes.c_char_p]
    lib.wbfbt_train_learned.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p]
    lib.wbfbt_status_string.argtypes = [i]
    lib.wbfbt_status_string.restype = ctypes.c_char_p
    return lib   # every other entry point returns int, ctypes' default


_LIB: ctypes.CDLL | None = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _check(status: int, what: str):
    if status != 0:
        raise WbfbtError(status, what)


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def default_opts() -> Opts:
    o = Opts()
    lib().wbfbt_default_opts(ctypes.byref(o))
    return o


def sinker_setup(nx: int, k: int, centres, omega: float, delta: float, dr: float, beta: float = 10.0,
                 ny: int | None = None, nz: int | None = None, lengths=(1.0, 1.0, 1.0), device="cuda"):
    """Multi-sinker viscosity and forcing of Sec. 2.1 at every node; returns (mu, f) device tensors."""
    ny, nz = ny or nx, nz or nx
    mesh = Mesh(nx, ny, nz, *lengths)
    nn = (k * nx + 1) * (k * ny + 1) * (k * nz + 1)
    mu = torch.empty(nn, dtype=torch.float64, device=device)
    f = torch.empty(3 * nn, dtype=torch.float64, device=device)
    c = torch.as_tensor(centres, dtype=torch.float64).contiguous().cpu()
    _check(lib().wbfbt_sinker_setup(ctypes.byref(mesh), k, ctypes.c_void_p(c.data_ptr()), int(c.shape[0]), omega,
                                    delta, dr, beta, _ptr(mu), _ptr(f), _stream()), "wbfbt_sinker_setup")
    return mu, f


def sinker_setup_at(X: torch.Tensor, nx: int, k: int, centres, omega: float, delta: float, dr: float,
                    beta: float = 10.0, ny: int | None = None, nz: int | None = None, lengths=(1.0, 1.0, 1.0)):
    """The fields of Sec. 2.1 at the node positions X (float64 device tensor [3][nodes])."""
    ny, nz = ny or nx, nz or nx
    mesh = Mesh(nx, ny, nz, *lengths)
    nn = (k * nx + 1) * (k * ny + 1) * (k * nz + 1)
    if X.dtype != torch.float64 or X.numel() != 3 * nn or not X.is_cuda:
        raise ValueError("X must be a float64 device tensor with 3 * n_nodes entries")
    X = X.contiguous()
    mu = torch.empty(nn, dtype=torch.float64, device=X.device)
    f = torch.empty(3 * nn, dtype=torch.float64, device=X.device)
    c = torch.as_tensor(centres, dtype=torch.float64).contiguous().cpu()
    _check(lib().wbfbt_sinker_setup_at(ctypes.byref(mesh), k, _ptr(X), ctypes.c_void_p(c.data_ptr()),
                                       int(c.shape[0]), omega, delta, dr, beta, _ptr(mu), _ptr(f), _stream()),
           "wbfbt_sinker_setup_at")
    return mu, f


def node_coords(nx: int, k: int, ny: int | None = None, nz: int | None = None, lengths=(1.0, 1.0, 1.0),
                device="cuda") -> torch.Tensor:
    """The brick's node positions, float64 device tensor [3][nodes] (component-major)."""
    ny, nz = ny or nx, nz or nx
    mesh = Mesh(nx, ny, nz, *lengths)
    X = torch.empty(3 * (k * nx + 1) * (k * ny + 1) * (k * nz + 1), dtype=torch.float64, device=device)
    _check(lib().wbfbt_node_coords(ctypes.byref(mesh), k, _ptr(X), _stream()), "wbfbt_node_coords")
    return X


def launch_count() -> int:
    """Kernels launched by libwbfbt.so so far in this process."""
    return lib().wbfbt_launch_count()


def apply_Kw_noalloc(nx: int, k: int, mu: torch.Tensor, a: float, p: torch.Tensor, y: torch.Tensor,
                     ny: int | None = None, nz: int | None = None, lengths=(1.0, 1.0, 1.0)) -> torch.Tensor:
    """y = B C^-1 B^T p without a context and without any device allocation (FP64 device tensors).

    For callers that cannot allocate device memory; the temporaries live in a static device
    array of the library (meshes up to NOALLOC_MAX_NODES velocity nodes).  Concurrent calls
    on one device race on that array.
    """
    mesh = Mesh(nx, ny or nx, nz or nx, *lengths)
    _check(lib().wbfbt_apply_Kw_noalloc(ctypes.byref(mesh), k, _ptr(mu), a, _ptr(p), _ptr(y), _stream()),
           "wbfbt_apply_Kw_noalloc")
    return y


@dataclass
class SolveResult:
    iters: int
    rel_res: float
    status: int


class Solver:
    """Owns one wbfbt_ctx.  All tensors are device tensors on the current stream unless noted."""

    def __init__(self, nx: int, k: int, mu: torch.Tensor, ny: int | None = None, nz: int | None = None,
                 lengths=(1.0, 1.0, 1.0), a_l: float = 1.0, a_r: float = 0.0, restart: int = 50,
                 cheb_degree: int = 3, mg_min_n: int = 4, precision: int = F64, schur_sign: int = -1,
                 use_graphs: bool = True, elem_kernels: int = 0, schur: int = SCHUR_WBFBT,
                 arnoldi_precision: int = F64, weights: int = WEIGHTS_SQRT_MU, kinv_cycles: int = 1,
                 ainv_cycles: int = 1,
                 pmg: bool = False):
        self.nx, self.ny, self.nz, self.k = nx, ny or nx, nz or nx, k
        self.mesh = Mesh(self.nx, self.ny, self.nz, *lengths)
        o = default_opts()
        o.a_l, o.a_r, o.restart, o.cheb_degree = a_l, a_r, restart, cheb_degree
        o.mg_min_n, o.precision, o.schur_sign, o.use_graphs = mg_min_n, precision, schur_sign, int(use_graphs)
        o.elem_kernels = elem_kernels
        o.schur = schur
        o.arnoldi_precision = arnoldi_precision
        o.weights = weights
        o.kinv_cycles = kinv_cycles
        o.ainv_cycles = ainv_cycles
        o.pmg = int(pmg)
        self.opts = o
        self.precision = precision
        self._mu = mu.contiguous()
        h = ctypes.c_void_p()
        _check(lib().wbfbt_create(ctypes.byref(self.mesh), k, _ptr(self._mu), ctypes.byref(o), _stream(),
                                  ctypes.byref(h)), "wbfbt_create")
        self.h = h
        nn, ne = ctypes.c_longlong(), ctypes.c_longlong()
        npe, nl = ctypes.c_int(), ctypes.c_int()
        _check(lib().wbfbt_sizes(h, ctypes.byref(nn), ctypes.byref(ne), ctypes.byref(npe), ctypes.byref(nl)),
               "wbfbt_sizes")
        self.n_nodes, self.n_elem, self.np, self.n_levels = nn.value, ne.value, npe.value, nl.value
        self.n_u, self.n_p = 3 * self.n_nodes, self.n_elem * self.np

    def setup(self, mu: torch.Tensor):
        """Re-run the viscosity-dependent setup for a new mu (no allocation)."""
        self._mu = mu.contiguous()
        _check(lib().wbfbt_setup(self.h, _ptr(self._mu)), "wbfbt_setup")

    def set_geometry(self, X: "torch.Tensor | None"):
        """Mapped hexahedra: X holds the nodal coordinates, component-major [3][nodes] float64
        (device or host), or None for the brick.  The operator applies, the Krylov operator and the
        load vector of solve() take the mapped geometry; the preconditioner stays the brick's."""
        if X is None:
            _check(lib().wbfbt_set_geometry(self.h, None), "wbfbt_set_geometry")
            self._X = None
            return
        if X.dtype != torch.float64 or X.numel() != self.n_u:
            raise ValueError("X must be float64 with 3 * n_nodes entries, component-major")
        self._X = X.contiguous()
        _check(lib().wbfbt_set_geometry(self.h, _ptr(self._X)), "wbfbt_set_geometry")

    def attach_net(self, net: "Net | None", which_mask: int = 2, accept_ratio: float = 1.0):
        """Use `net` for K_r (bit 1) and/or K_l (bit 0) inside S~^-1, V-cycle as fallback.

        A learned step is kept only if it leaves ||r - K_w z|| < accept_ratio ||r||.
        """
        _check(lib().wbfbt_attach_net(self.h, net.h if net is not None else None, which_mask, accept_ratio),
               "wbfbt_attach_net")
        self._net = net

    def learned_sample(self, which: int, r: torch.Tensor):
        """(features [E][1+Np], target [E][Np]) for pressure residual r (FP64 device, mean-free)."""
        x = torch.empty((self.n_elem, 1 + self.np), dtype=torch.float32, device=r.device)
        y = torch.empty((self.n_elem, self.np), dtype=torch.float32, device=r.device)
        _check(lib().wbfbt_learned_sample(self.h, which, _ptr(r), _ptr(x), _ptr(y)), "wbfbt_learned_sample")
        return x, y

    def load_learned(self, path: str):
        """Load a checkpoint into a network owned by the context and attach it for K_r."""
        _check(lib().wbfbt_load_learned(self.h, str(path).encode()), "wbfbt_load_learned")

    def train_learned(self, out_path: str, **cfg):
        """Train the learned correction in the library (keys: fields, per_field, epochs, batch,
        lr, seed, init_seed, omega, delta) and write the checkpoint to out_path."""
        js = json.dumps(cfg).encode() if cfg else None
        _check(lib().wbfbt_train_learned(self.h, js, str(out_path).encode()), "wbfbt_train_learned")

    def learned_stats(self):
        a, r = ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().wbfbt_learned_stats(self.h, ctypes.byref(a), ctypes.byref(r)), "wbfbt_learned_stats")
        return a.value, r.value

    def close(self):
        if getattr(self, "h", None):
            lib().wbfbt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def device_bytes(self) -> int:
        return lib().wbfbt_device_bytes(self.h)

    @property
    def pdtype(self) -> torch.dtype:
        return torch.float64 if self.precision == F64 else torch.float32

    def _apply(self, name, x, nout, *extra):
        y = torch.empty(nout, dtype=x.dtype, device=x.device)
        _check(getattr(lib(), name)(self.h, *extra, _ptr(x), _ptr(y), _dtype_code(x)), name)
        return y

    def apply_A(self, u):
        return self._apply("wbfbt_apply_A", u, self.n_u)

    def apply_B(self, u):
        return self._apply("wbfbt_apply_B", u, self.n_p)

    def apply_BT(self, p):
        return self._apply("wbfbt_apply_BT", p, self.n_u)

    def apply_K(self, x):
        return self._apply("wbfbt_apply_K", x, self.n_u + self.n_p)

    def apply_Kw(self, which: int, p):
        return self._apply("wbfbt_apply_Kw", p, self.n_p, which)

    def apply_Ainv(self, r):
        return self._apply("wbfbt_apply_Ainv", r, self.n_u)

    def apply_Kinv(self, which: int, r):
        return self._apply("wbfbt_apply_Kinv", r, self.n_p, which)

    def apply_schur_inv(self, r):
        return self._apply("wbfbt_apply_schur_inv", r, self.n_p)

    def apply_precond(self, x):
        return self._apply("wbfbt_apply_precond", x, self.n_u + self.n_p)

    def solve_block(self, block: int, b: torch.Tensor, rtol: float = 1e-6, maxit: int = 1000, check=True):
        """One preconditioner block alone (BLOCK_A, BLOCK_KL, BLOCK_KR) with FGMRES and its V-cycle."""
        b = b.contiguous()
        x = torch.empty_like(b)
        its, rel = ctypes.c_int(), ctypes.c_double()
        st = lib().wbfbt_solve_block(self.h, block, _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(its), ctypes.byref(rel))
        if check and st not in (0, -5):
            _check(st, "wbfbt_solve_block")
        return x, SolveResult(its.value, rel.value, st)

    def solve(self, f: torch.Tensor, rtol: float = 1e-6, maxit: int = 1000, u=None, p=None, check=True):
        """Solve with body force f [3][nodes] (device or pinned/pageable host float64 tensor)."""
        dev = f.device
        u = torch.empty(self.n_u, dtype=torch.float64, device=dev) if u is None else u
        p = torch.empty(self.n_p, dtype=torch.float64, device=dev) if p is None else p
        its, rel = ctypes.c_int(), ctypes.c_double()
        st = lib().wbfbt_solve(self.h, _ptr(f), _ptr(u), _ptr(p), rtol, maxit, ctypes.byref(its), ctypes.byref(rel))
        if check and st not in (0, -5):
            _check(st, "wbfbt_solve")
        return u, p, SolveResult(its.value, rel.value, st)


class Net:
    """The learned pressure-Poisson correction (a BF16 tensor-core U-Net), owning a wbfbt_net."""

    def __init__(self, cin: int, cout: int, n: int, max_batch: int = 1):
        self.cin, self.cout, self.n, self.max_batch = cin, cout, n, max_batch
        h = ctypes.c_void_p()
        _check(lib().wbfbt_net_create(cin, cout, n, max_batch, _stream(), ctypes.byref(h)), "wbfbt_net_create")
        self.h = h
        self.n_params = lib().wbfbt_net_param_count(h)

    @staticmethod
    def num_params(cin: int, cout: int) -> int:
        return lib().wbfbt_net_num_params(cin, cout)

    def set_params(self, theta: torch.Tensor):
        theta = theta.to(torch.float32).contiguous()
        _check(lib().wbfbt_net_set_params(self.h, _ptr(theta)), "wbfbt_net_set_params")
        torch.cuda.synchronize()

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(lib().wbfbt_net_get_params(self.h, _ptr(out)), "wbfbt_net_get_params")
        return out

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        x = x.contiguous()
        batch = x.shape[0] if x.dim() == 3 else 1
        y = torch.empty((batch, self.n ** 3, self.cout), dtype=torch.float32, device=x.device)
        _check(lib().wbfbt_net_forward(self.h, _ptr(x), batch, _ptr(y)), "wbfbt_net_forward")
        return y

    def loss_grad(self, x: torch.Tensor, target: torch.Tensor, want_grad: bool = True):
        x, target = x.contiguous(), target.contiguous()
        batch = x.shape[0] if x.dim() == 3 else 1
        loss = ctypes.c_double()
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device) if want_grad else None
        _check(lib().wbfbt_net_loss_grad(self.h, _ptr(x), _ptr(target), batch, ctypes.byref(loss),
                                         _ptr(g) if g is not None else None), "wbfbt_net_loss_grad")
        return loss.value, g

    def conv_layer(self, layer: int, n: int, x: torch.Tensor, g: torch.Tensor | None = None,
                   cout: int | None = None, want_y: bool = True):
        """One layer in isolation: (y [batch][n^3][cout], dW [27][cin][cout] or None)."""
        x = x.contiguous()
        batch = x.shape[0]
        y = torch.empty((batch, n ** 3, cout), dtype=torch.float32, device=x.device) if want_y else None
        dw = None
        if g is not None:
            g = g.contiguous()
            dw = torch.empty((27, x.shape[-1], g.shape[-1]), dtype=torch.float32, device=x.device)
        _check(lib().wbfbt_net_conv_layer(self.h, layer, n, batch, _ptr(x), _ptr(y) if y is not None else None,
                                          _ptr(g) if g is not None else None, _ptr(dw) if dw is not None else None),
               "wbfbt_net_conv_layer")
        return y, dw

    def adam_step(self, lr: float):
        _check(lib().wbfbt_net_adam_step(self.h, lr), "wbfbt_net_adam_step")

    def save(self, path: str):
        _check(lib().wbfbt_net_save(self.h, path.encode()), "wbfbt_net_save")

    def load(self, path: str):
        _check(lib().wbfbt_net_load(self.h, path.encode()), "wbfbt_net_load")

    def close(self):
        if getattr(self, "h", None):
            lib().wbfbt_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
