"""ctypes binding of librdg.so (argument marshalling only; every computation runs in the
library's sm_103a kernels).  Device memory and streams come from PyTorch.

The low-level functions keep the C names (``rdg_rhs_eval`` ...); :class:`Solver` wraps one
context.  There is no CPU fallback: if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "librdg.so")

RDG_OK, RDG_EINVAL, RDG_ENOMEM, RDG_ECUDA, RDG_EMESH, RDG_ERANK, RDG_ETIMEOUT, RDG_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
BC_PERIODIC, BC_DIRICHLET = 0, 1
FP64, FP32, FP32_3XTF32 = 0, 1, 2
TAU_CONST, TAU_COS, TAU_SIN = 0, 1, 2
IFACE_ALG2, IFACE_HARMONIC, IFACE_ALG1 = 0, 1, 2
SSP_RK3, LSRK54 = 0, 1
STAGE_AUTO, STAGE_TWO_KERNELS, STAGE_ONE_KERNEL = 0, 1, 2
BATCH_AUTO, BATCH_GRAPH, BATCH_PERSISTENT = 0, 1, 2
ERR_NAMES = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EMESH", -5: "ERANK", -6: "ETIMEOUT", -7: "ESTATE"}

# symbol -> (restype, argtypes)
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double
_INT = ctypes.c_int
SIGNATURES = {
    "rdg_version": (ctypes.c_char_p, []),
    "rdg_last_error": (ctypes.c_char_p, [_P]),
    "rdg_create": (_INT, [ctypes.POINTER(_P), _INT, _P]),
    "rdg_destroy": (_INT, [_P]),
    "rdg_mesh_upload": (_INT, [_P, _I64, _P, _I64, _P, _I32, _P]),
    "rdg_mesh_upload_partition": (_INT, [_P, _I64, _P, _I64, _P, _I32, _P, _I64]),
    "rdg_rk_stage": (_INT, [_P, _INT, _D, _D]),
    "rdg_stage_buffer": (_INT, [_P, _INT, ctypes.POINTER(_P)]),
    "rdg_rows_gather": (_INT, [_P, _P, _P, _I64, _P]),
    "rdg_rows_scatter": (_INT, [_P, _P, _P, _I64, _P]),
    "rdg_operator_setup": (_INT, [_P, _INT, _P, _D, _D, _INT, _INT]),
    "rdg_operator_setup_aniso": (_INT, [_P, _INT, _P, _P, _D, _D, _INT, _INT]),
    "rdg_operator_setup_nodal": (_INT, [_P, _INT, _P, _D, _D, _INT, _INT]),
    "rdg_set_forcing": (_INT, [_P, _INT, _P, _P, _P, _INT, _P, _P, _P]),
    "rdg_mesh_counts": (_INT, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "rdg_get_node_coords": (_INT, [_P, _P]),
    "rdg_get_ghost_coords": (_INT, [_P, _P]),
    "rdg_set_state": (_INT, [_P, _P, _INT]),
    "rdg_get_state": (_INT, [_P, _P, _INT]),
    "rdg_rhs_eval": (_INT, [_P, _P, _P, _D]),
    "rdg_rhs_eval_static": (_INT, [_P, _P, _P, _D]),
    "rdg_rk_step": (_INT, [_P, _D, _D]),
    "rdg_solve_to_time": (_INT, [_P, _D, _D, _I64]),
    "rdg_synchronize": (_INT, [_P]),
    "rdg_profile": (_INT, [_P, _INT]),
    "rdg_set_l2_resident_bytes": (_INT, [_P, _I64]),
    "rdg_kernel_stats": (_INT, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_D), _INT]),
    "rdg_query_bytes": (_INT, [_INT, _I64, _I64, _I64, _INT, _INT, _INT, ctypes.POINTER(_I64)]),
    "rdg_reference_operator": (_INT, [_INT, _INT, _P]),
    "rdg_get_edge_operators": (_INT, [_P, _P, _P]),
    "rdg_set_integrator": (_INT, [_P, _INT]),
    "rdg_rk_stage_part": (_INT, [_P, _INT, _INT, _D, _D]),
    "rdg_split_counts": (_INT, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "rdg_set_stage_form": (_INT, [_P, _INT]),
    "rdg_gemm_hold_tile": (_INT, [_P, ctypes.c_int64]),
    "rdg_get_stage_form": (_INT, [_P, ctypes.POINTER(ctypes.c_int)]),
    "rdg_error_quadrature": (_INT, [_P, ctypes.POINTER(_INT), _P]),
    "rdg_error_norms": (_INT, [_P, _P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "rdg_peak_fma": (_INT, [_INT, _INT, ctypes.POINTER(_D)]),
    "rdg_stream_read": (_INT, [_INT, _I64, ctypes.POINTER(_D)]),
    "rdg_batch_create": (_INT, [ctypes.POINTER(_P), _INT, _P, _INT]),
    "rdg_batch_destroy": (_INT, [_P]),
    "rdg_batch_last_error": (ctypes.c_char_p, [_P]),
    "rdg_batch_add": (_INT, [_P, _P, _D, _D]),
    "rdg_batch_remove": (_INT, [_P, _P]),
    "rdg_batch_size": (_INT, [_P, ctypes.POINTER(_INT)]),
    "rdg_batch_set_chunk": (_INT, [_P, _INT]),
    "rdg_batch_step": (_INT, [_P, _I64]),
    "rdg_batch_synchronize": (_INT, [_P]),
    "rdg_batch_set_mode": (_INT, [_P, _INT]),
    "rdg_batch_get_mode": (_INT, [_P, ctypes.POINTER(_INT)]),
    "rdg_batch_set_tiles": (_INT, [_P, _INT, _INT, _INT]),
    "rdg_batch_set_wait_limit": (_INT, [_P, _D]),
    "rdg_batch_hold_phase": (_INT, [_P, _INT, _I64]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load librdg.so (raises if it was not built) and declare every C signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("librdg.so not built (%s): run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("rdg error %s (%d): %s" % (ERR_NAMES.get(code, "?"), code, msg))
        self.code = code


def _check(rc, ctx=None):
    if rc != RDG_OK:
        msg = load().rdg_last_error(ctx)
        raise RdgError(rc, msg.decode() if msg else "")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def np_of(N):
    return (N + 1) * (N + 2) // 2


def query_bytes(N, nt, n_edges, n_boundary, precision, nsrc=0, nghost=0):
    out = _I64(0)
    _check(load().rdg_query_bytes(N, nt, n_edges, n_boundary, precision, nsrc, nghost, ctypes.byref(out)))
    return out.value


def peak_fma(device=0, precision=FP32):
    """FMA rate of the device in FLOP/s (rdg_peak_fma)."""
    out = _D(0.0)
    _check(load().rdg_peak_fma(device, precision, ctypes.byref(out)))
    return out.value


def stream_read_seconds(device=0, nbytes=1 << 30):
    """Time of a plain streaming read of nbytes from device memory (rdg_stream_read)."""
    out = _D(0.0)
    _check(load().rdg_stream_read(device, int(nbytes), ctypes.byref(out)))
    return out.value


def reference_operator(N, which):
    Np, Nfp, Mp = np_of(N), N + 1, (N + 1) ** 2
    shape = {0: (2, Np), 1: (Np, Np), 2: (Np, Np), 3: (Np, 3 * Nfp), 4: (Mp, 2 * Np), 5: (Np, Np),
             6: (2, Np, Nfp, 2, Np), 7: (3, Np), 8: (Nfp,), 9: (2, Nfp, Np), 10: (2, 2, Np, Np),
             11: (2, 2, Np, Np)}[which]
    out = np.zeros(shape)
    _check(load().rdg_reference_operator(N, which, _ptr(out)))
    return out


class Solver:
    """One library context: mesh, operators of order N and the resident state."""

    def __init__(self, xy, tri, N: int, D_elem, v=(0.0, 0.0), bc: int = BC_PERIODIC, period=(1.0, 1.0),
                 precision: int = FP32, device: int = 0, stream=None, interface: int = IFACE_ALG2,
                 n_owned: Optional[int] = None):
        import torch
        self.torch = torch
        self.lib = load()
        self.device = device
        self.N, self.Np, self.Nfp = N, np_of(N), N + 1
        self.precision = precision
        self.dtype = torch.float64 if precision == FP64 else torch.float32   # FP32 and FP32_3XTF32
        self.np_dtype = np.float64 if precision == FP64 else np.float32
        self.stream, handle = _stream_handle(torch, stream, device)
        ctx = _P()
        _check(self.lib.rdg_create(ctypes.byref(ctx), device, _P(handle)))
        self.ctx = ctx
        xy = np.ascontiguousarray(xy, np.float64)
        tri = np.ascontiguousarray(tri, np.int32)
        per = np.ascontiguousarray(period if period is not None else (0.0, 0.0), np.float64)
        if n_owned is None:
            self._call("rdg_mesh_upload", xy.shape[0], _ptr(xy), tri.shape[0], _ptr(tri), bc,
                       _ptr(per) if period is not None else None)
        else:   # one part of a mesh split across ranks: triangles n_owned.. are halo copies
            self._call("rdg_mesh_upload_partition", xy.shape[0], _ptr(xy), tri.shape[0], _ptr(tri), bc,
                       _ptr(per) if period is not None else None, int(n_owned))
        self.n_owned = tri.shape[0] if n_owned is None else int(n_owned)
        Da = np.asarray(D_elem, np.float64)
        if Da.ndim == 2 and Da.shape[1] == self.Np:     # [nt, Np]: D given at the nodes
            Dn = np.ascontiguousarray(Da)
            self._call("rdg_operator_setup_nodal", N, _ptr(Dn), float(v[0]), float(v[1]), precision, interface)
        elif Da.ndim == 2:        # [nt, 2]: the diagonal tensor (Dx, Dy)
            Dx = np.ascontiguousarray(Da[:, 0])
            Dy = np.ascontiguousarray(Da[:, 1])
            self._call("rdg_operator_setup_aniso", N, _ptr(Dx), _ptr(Dy), float(v[0]), float(v[1]), precision,
                       interface)
        else:
            D = np.ascontiguousarray(np.broadcast_to(Da, (tri.shape[0],)))
            self._call("rdg_operator_setup", N, _ptr(D), float(v[0]), float(v[1]), precision, interface)
        K, E, B = _I64(), _I64(), _I64()
        self._call("rdg_mesh_counts", ctypes.byref(K), ctypes.byref(E), ctypes.byref(B))
        self.K, self.E, self.B = K.value, E.value, B.value

    def _call(self, name, *args):
        _check(getattr(self.lib, name)(self.ctx, *args), self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.rdg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- geometry ---------------------------------------------------------------------
    def node_coords(self):
        out = np.zeros((self.K, self.Np, 2))
        self._call("rdg_get_node_coords", _ptr(out))
        return out

    def ghost_coords(self):
        out = np.zeros((self.B, self.Np, 2))
        self._call("rdg_get_ghost_coords", _ptr(out) if self.B else None)
        return out

    def edge_operators(self):
        W = np.zeros((self.E, self.Nfp, 2 * self.Np))
        ids = np.zeros((self.E, 4), np.int32)
        self._call("rdg_get_edge_operators", _ptr(W), _ptr(ids))
        return W, ids

    # -- forcing ----------------------------------------------------------------------
    def set_forcing(self, src: Sequence = (), ghost: Sequence = ()):
        """src: [(S nodal [K, Np], kind, omega)], ghost: [(G [B, Np] at ghost nodes, kind, omega)]."""
        S = np.ascontiguousarray(np.stack([np.asarray(s[0], np.float64) for s in src])) if src else None
        sk = np.array([s[1] for s in src], np.int32)
        so = np.array([s[2] for s in src], np.float64)
        G = np.ascontiguousarray(np.stack([np.asarray(g[0], np.float64) for g in ghost])) if ghost else None
        gk = np.array([g[1] for g in ghost], np.int32)
        go = np.array([g[2] for g in ghost], np.float64)
        self._call("rdg_set_forcing", len(src), _ptr(S) if S is not None else None, _ptr(sk), _ptr(so),
                   len(ghost), _ptr(G) if G is not None else None, _ptr(gk), _ptr(go))

    # -- state and stepping ----------------------------------------------------------
    def _dev_tensor(self, t):
        torch = self.torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype and t.is_contiguous()
                and t.numel() == self.K * self.Np):
            raise ValueError("expected a contiguous CUDA %s tensor of %d values" % (self.dtype, self.K * self.Np))
        return _P(t.data_ptr())

    def new_field(self):
        return self.torch.zeros((self.K, self.Np), dtype=self.dtype, device="cuda:%d" % self.device)

    def _host_tensor(self, t):
        torch = self.torch
        if not (t.dtype == self.dtype and t.is_contiguous() and t.numel() == self.K * self.Np):
            raise ValueError("expected a contiguous host %s tensor of %d values" % (self.dtype, self.K * self.Np))
        return _P(t.data_ptr())

    def set_state(self, u):
        """From a NumPy array or a host tensor (pinned memory copies fastest), or a CUDA tensor."""
        if isinstance(u, np.ndarray):
            a = np.ascontiguousarray(u, self.np_dtype)
            self._call("rdg_set_state", _ptr(a), 0)
        elif not u.is_cuda:
            self._call("rdg_set_state", self._host_tensor(u), 0)
        else:
            self._call("rdg_set_state", self._dev_tensor(u), 1)

    def get_state(self, out=None):
        """Into `out`: a CUDA tensor (a new one if None) or a host tensor (e.g. pinned)."""
        if out is None:
            out = self.new_field()
        if out.is_cuda:
            self._call("rdg_get_state", self._dev_tensor(out), 1)
        else:
            self._call("rdg_get_state", self._host_tensor(out), 0)
        return out

    def get_state_host(self):
        a = np.zeros((self.K, self.Np), self.np_dtype)
        self._call("rdg_get_state", _ptr(a), 0)
        return a

    def rhs_eval(self, u, rhs, t: float = 0.0):
        self._call("rdg_rhs_eval", self._dev_tensor(u), self._dev_tensor(rhs), float(t))

    def rk_step(self, t: float, dt: float):
        self._call("rdg_rk_step", float(t), float(dt))

    def rk_stage(self, stage: int, t: float, dt: float):
        """One stage of a step from step start t (rdg_rk_stage)."""
        self._call("rdg_rk_stage", int(stage), float(t), float(dt))

    def rk_stage_part(self, stage: int, part: int, t: float, dt: float):
        """Part 0 or 1 of a stage, around a halo exchange (rdg_rk_stage_part)."""
        self._call("rdg_rk_stage_part", int(stage), int(part), float(t), float(dt))

    def split_counts(self):
        """(owned elements, e_split): edges [0, e_split) touch no halo element."""
        n, e = ctypes.c_int64(0), ctypes.c_int64(0)
        self._call("rdg_split_counts", ctypes.byref(n), ctypes.byref(e))
        return n.value, e.value

    def stage_buffer(self, stage: int) -> int:
        """Device address of the input buffer of `stage` (rdg_stage_buffer)."""
        p = _P()
        self._call("rdg_stage_buffer", int(stage), ctypes.byref(p))
        return p.value

    def rows_gather(self, src: int, idx, n: int, dst: int):
        """dst[i] = src[idx[i]] for i < n (device addresses; idx a CUDA int32 tensor)."""
        self._call("rdg_rows_gather", _P(src), _P(idx.data_ptr()), int(n), _P(dst))

    def rows_scatter(self, src: int, idx, n: int, dst: int):
        """dst[idx[i]] = src[i] for i < n (device addresses; idx a CUDA int32 tensor)."""
        self._call("rdg_rows_scatter", _P(src), _P(idx.data_ptr()), int(n), _P(dst))

    def set_integrator(self, kind: int):
        """SSP_RK3 (default) or LSRK54 (the paper's five-stage fourth-order scheme)."""
        self._call("rdg_set_integrator", int(kind))

    def set_stage_form(self, form: int):
        """STAGE_AUTO (default), STAGE_TWO_KERNELS or STAGE_ONE_KERNEL (rdg_set_stage_form)."""
        self._call("rdg_set_stage_form", int(form))

    def gemm_hold_tile(self, tile: int):
        """Test hook: GEMM-form edge tile `tile` is never released (-1: none)."""
        self._call("rdg_gemm_hold_tile", int(tile))

    @property
    def stage_form(self) -> int:
        """The kernel form a right-hand-side stage uses (STAGE_ONE_KERNEL or STAGE_TWO_KERNELS)."""
        f = ctypes.c_int(0)
        self._call("rdg_get_stage_form", ctypes.byref(f))
        return f.value

    def solve_to_time(self, t0: float, dt: float, nsteps: int):
        self._call("rdg_solve_to_time", float(t0), float(dt), int(nsteps))

    def synchronize(self):
        self._call("rdg_synchronize")

    def set_l2_resident_bytes(self, nbytes: int):
        """Operator bytes kept L2-resident across stages (-1 default = 0 = none); speed only."""
        self._call("rdg_set_l2_resident_bytes", int(nbytes))

    def profile(self, enable: bool = True):
        self._call("rdg_profile", 1 if enable else 0)

    # -- error norms (FP64 on the GPU) -------------------------------------------------
    def error_quadrature(self):
        """Physical coordinates [K, nq, 2] of the error norms' quadrature points."""
        nq = _INT(0)
        self._call("rdg_error_quadrature", ctypes.byref(nq), None)
        out = np.zeros((self.K, nq.value, 2))
        self._call("rdg_error_quadrature", ctypes.byref(nq), _ptr(out))
        return out

    def error_norms(self, exact_q, u=None):
        """(L2, L_inf of cell means) of u (a CUDA tensor; None: the resident state) against
        the exact values at the error_quadrature points (array or CUDA tensor [K, nq])."""
        torch = self.torch
        ue = exact_q if isinstance(exact_q, torch.Tensor) else torch.tensor(np.asarray(exact_q, np.float64))
        ue = ue.to(device="cuda:%d" % self.device, dtype=torch.float64).contiguous()
        l2, li = _D(0.0), _D(0.0)
        self._call("rdg_error_norms", self._dev_tensor(u) if u is not None else None, _P(ue.data_ptr()),
                   ctypes.byref(l2), ctypes.byref(li))
        return l2.value, li.value

    def kernel_stats(self, reset: bool = True):
        """{'edge': (launches, ms), 'elem': (launches, ms)} of the event-timed launches."""
        n = (_I64 * 2)()
        ms = (_D * 2)()
        self._call("rdg_kernel_stats", n, ms, 1 if reset else 0)
        return {"edge": (n[0], ms[0]), "elem": (n[1], ms[1])}


def _stream_handle(torch, stream, device):
    if stream is None:
        stream = torch.cuda.current_stream(device)
    handle = stream.cuda_stream
    # torch's default stream (handle 0) is the legacy default stream, cudaStreamLegacy
    return stream, (handle if handle != 0 else 1)


class Batch:
    """Independent solves stepped together: each member is a :class:`Solver` with its own
    mesh, order, precision and dt; :meth:`step` advances all of them by the same number of
    SSP-RK3 steps with one CUDA-graph launch per chunk of steps."""

    def __init__(self, device: int = 0, stream=None, chunk: int = 16):
        import torch
        self.torch = torch
        self.lib = load()
        self.device = device
        self.stream, handle = _stream_handle(torch, stream, device)
        b = _P()
        rc = self.lib.rdg_batch_create(ctypes.byref(b), device, _P(handle), int(chunk))
        if rc != RDG_OK:
            raise RdgError(rc, "rdg_batch_create failed")
        self.b = b
        self.members = []

    def _call(self, name, *args):
        rc = getattr(self.lib, name)(self.b, *args)
        if rc != RDG_OK:
            msg = self.lib.rdg_batch_last_error(self.b)
            raise RdgError(rc, msg.decode() if msg else "")

    def add(self, solver: "Solver", dt: float, t0: float = 0.0):
        self._call("rdg_batch_add", solver.ctx, float(t0), float(dt))
        self.members.append(solver)

    def remove(self, solver: "Solver"):
        self._call("rdg_batch_remove", solver.ctx)
        self.members.remove(solver)

    def __len__(self):
        n = _INT(0)
        self._call("rdg_batch_size", ctypes.byref(n))
        return n.value

    def step(self, nsteps: int):
        self._call("rdg_batch_step", int(nsteps))

    def set_chunk(self, chunk: int):
        """Steps per replayed graph (the graph is captured again on the next step)."""
        self._call("rdg_batch_set_chunk", int(chunk))

    def synchronize(self):
        self._call("rdg_batch_synchronize")

    def set_mode(self, mode: int):
        """BATCH_AUTO (default), BATCH_GRAPH or BATCH_PERSISTENT."""
        self._call("rdg_batch_set_mode", int(mode))

    @property
    def mode(self) -> int:
        m = _INT(0)
        self._call("rdg_batch_get_mode", ctypes.byref(m))
        return m.value

    def set_tiles(self, N: int, edges_per_thread: int, tiles_per_item: int = 1):
        self._call("rdg_batch_set_tiles", int(N), int(edges_per_thread), int(tiles_per_item))

    def set_wait_limit(self, seconds: float):
        self._call("rdg_batch_set_wait_limit", float(seconds))

    def hold_phase(self, member: int, phase: int):
        """Test hook: phase `phase` of member `member` is never released (-1: no hold)."""
        self._call("rdg_batch_hold_phase", int(member), int(phase))

    def close(self):
        if getattr(self, "b", None):
            self.lib.rdg_batch_destroy(self.b)
            self.b = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
