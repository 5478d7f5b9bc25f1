"""Python front end of librlb: one relativistic lattice Boltzmann lattice on one GPU.

``RLB`` owns a librlb context whose device workspace is a torch tensor (the
caching allocator provides the memory, torch's current stream orders the
work).  Every method marshals arguments to the C entry point of the same name
in ``_native``; the computation runs in the library's CUDA kernels only.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _native as N

_PREC = {"fp64": N.RLB_FP64, "fp32": N.RLB_FP32_DEV, "fp32dev": N.RLB_FP32_DEV}
_EOS = {"ultra": N.RLB_EOS_ULTRA, "gamma_law": N.RLB_EOS_GAMMA_LAW}
_XBC = {"periodic": N.RLB_BC_PERIODIC, "inflow_outflow": N.RLB_BC_INFLOW_OUTFLOW,
        "outflow_both": N.RLB_BC_OUTFLOW_BOTH}
_ZBC = {"periodic": N.RLB_ZBC_PERIODIC, "halo": N.RLB_ZBC_HALO}


def _require_cuda(device):
    if not torch.cuda.is_available():
        raise RuntimeError("librlb needs a CUDA GPU; there is no CPU path")
    return torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())


class RLB:
    """A D3Q19 relativistic lattice Boltzmann lattice (f and g populations) on one GPU."""

    def __init__(self, nx, ny, nz, tau, c_l=1.0, precision="fp64", xbc="periodic", n_in=1.0, eps_in=1.0,
                 beta_in=(0.0, 0.0, 0.0), n_ref=1.0, eps_ref=1.0, device=None, stream=None, eos="ultra",
                 eos_gamma=4.0 / 3.0, eos_mass=0.0, zbc="periodic"):
        self.device = _require_cuda(device)
        prec = _PREC[precision] if isinstance(precision, str) else int(precision)
        x = _XBC[xbc] if isinstance(xbc, str) else int(xbc)
        e = _EOS[eos] if isinstance(eos, str) else int(eos)
        z = _ZBC[zbc] if isinstance(zbc, str) else int(zbc)
        self.params = N.make_params(nx, ny, nz, tau, c_l, prec, x, n_in, eps_in, beta_in, n_ref, eps_ref, e,
                                    eos_gamma, eos_mass, z)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.precision = "fp64" if prec == N.RLB_FP64 else "fp32"
        self.dtype = torch.float64 if prec == N.RLB_FP64 else torch.float32
        self.plane_stride, self.elem_bytes, self.state_bytes = N.rlb_state_layout(self.params)
        self.ws_bytes = N.rlb_workspace_bytes(self.params)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
            if self.stream != torch.cuda.current_stream(self.device):
                # the workspace is used on the context's stream: its memory is
                # reused only after that stream's work when it is freed
                self.ws.record_stream(self.stream)
            self.ctx = N.rlb_create(self.params, self.stream.cuda_stream, self.ws, self.ws_bytes)

    @staticmethod
    def reference_value(values) -> float:
        """Uniform FP32 deviation reference for a positive field: the value r that
        minimises the largest relative deviation max |v - r| / v over the field,
        r = 2 v_min v_max / (v_min + v_max).  Binary32 rounds the stored deviation
        v - r, so this bounds the relative rounding of every cell by the same
        factor on both ends of the range."""
        v = np.asarray(values, dtype=np.float64)
        lo, hi = float(v.min()), float(v.max())
        return 2.0 * lo * hi / (lo + hi)

    @classmethod
    def from_workload(cls, w, precision="fp64", device=None, n_ref=None, eps_ref=None, **kw):
        """Context for a ``workloads.Workload``; the FP32 reference defaults to
        ``reference_value`` of the initial fields over the non-solid cells (and the
        inflow state)."""
        m = np.ones(w.eps.shape, bool) if w.solid is None else (w.solid == 0)
        if n_ref is None:
            n_ref = cls.reference_value(np.append(w.n[m], w.n_in))
        if eps_ref is None:
            eps_ref = cls.reference_value(np.append(w.eps[m], w.eps_in))
        xbc = {0: "periodic", 1: "inflow_outflow", 2: "outflow_both"}[w.xbc]
        eos = dict(eos=getattr(w, "eos", 0), eos_gamma=getattr(w, "eos_gamma", 4.0 / 3.0),
                   eos_mass=getattr(w, "eos_mass", 0.0))
        eos.update(kw)
        return cls(w.nx, w.ny, w.nz, w.tau, w.c_l, precision, xbc, w.n_in, w.eps_in, w.beta_in, n_ref, eps_ref,
                   device=device, **eos)

    # -- memory ---------------------------------------------------------------
    def new_state(self) -> torch.Tensor:
        """A state-layout device buffer (38 planes of plane_stride elements)."""
        return torch.empty((38, self.plane_stride), dtype=self.dtype, device=self.device)

    def _view(self, ptr: int) -> torch.Tensor:
        off = ptr - self.ws.data_ptr()
        assert 0 <= off and off + self.state_bytes <= self.ws_bytes
        return self.ws[off:off + self.state_bytes].view(self.dtype).view(38, self.plane_stride)

    def state(self) -> torch.Tensor:
        """View of the context's current state (valid until the next step)."""
        return self._view(N.rlb_state_ptr(self.ctx))

    # -- forward --------------------------------------------------------------
    def init_fields(self, n, eps, beta, solid=None):
        """Initial fields as torch tensors on the device (float64; solid uint8)
        or numpy arrays on the host; n, eps (nz, ny, nx), beta (3, nz, ny, nx)."""
        if isinstance(n, torch.Tensor):
            args = [t.contiguous() for t in (n, eps, beta)]
            for t in args:
                assert t.dtype == torch.float64 and t.device == self.device and t.numel() in (self.N, 3 * self.N)
            s = None if solid is None else solid.to(self.device, torch.uint8).contiguous()
            with torch.cuda.device(self.device):
                N.rlb_init_fields(self.ctx, *args, s, N.RLB_DEVICE)
            self._keep = (args, s)
        else:
            args = [np.ascontiguousarray(a, dtype=np.float64) for a in (n, eps, beta)]
            s = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8)
            with torch.cuda.device(self.device):
                N.rlb_init_fields(self.ctx, *args, s, N.RLB_HOST)
        return self

    def step(self, nsteps: int = 1):
        N.rlb_step(self.ctx, nsteps)
        return self

    def step_into(self, src: torch.Tensor, dst: torch.Tensor, counted: bool = False):
        """One step from src into dst (caller states); counted=True adds it to
        the context's statistics as its next step."""
        (N.rlb_step_into_counted if counted else N.rlb_step_into)(self.ctx, src, dst)

    def save_state(self, dst: torch.Tensor):
        N.rlb_save_state(self.ctx, dst)

    def load_state(self, src: torch.Tensor):
        N.rlb_load_state(self.ctx, src)

    # -- checkpoint / resume through a host file ------------------------------
    CHECKPOINT_FORMAT = "rlb-state-v1"

    def _param_dict(self) -> dict:
        out = {}
        for name, _ in self.params._fields_:
            v = getattr(self.params, name)
            out[name] = list(v) if name == "beta_in" else v
        return out

    def save(self, path: str):
        """Write the current state to a file: one JSON header line (every
        rlb_params field, the layout, the steps taken) followed by the 38
        planes as raw little-endian values of the state's element type.
        ``load`` on a context with the same parameters resumes from it."""
        import json

        self.sync()
        hdr = {"format": self.CHECKPOINT_FORMAT, "params": self._param_dict(), "plane_stride": self.plane_stride,
               "elem_bytes": self.elem_bytes, "steps": self.stats()["steps"]}
        data = self.state().detach().cpu().numpy()
        with open(path, "wb") as fh:
            fh.write((json.dumps(hdr) + "\n").encode())
            fh.write(data.astype(data.dtype.newbyteorder("<"), copy=False).tobytes())
        return self

    def load(self, path: str):
        """Resume from a file written by ``save``: the parameters and the layout
        must match this context's (ValueError otherwise)."""
        import json

        with open(path, "rb") as fh:
            hdr = json.loads(fh.readline().decode())
            raw = fh.read()
        if hdr.get("format") != self.CHECKPOINT_FORMAT:
            raise ValueError(f"not an RLB state file: {path}")
        if hdr["params"] != self._param_dict():
            raise ValueError("the state file was written with other parameters")
        if hdr["plane_stride"] != self.plane_stride or hdr["elem_bytes"] != self.elem_bytes:
            raise ValueError("the state file has another layout")
        dt = np.dtype("<f8" if self.elem_bytes == 8 else "<f4")
        arr = np.frombuffer(raw, dtype=dt)
        if arr.size != 38 * self.plane_stride:
            raise ValueError("truncated state file")
        t = torch.from_numpy(arr.reshape(38, self.plane_stride).astype(dt.newbyteorder("="))).to(self.device)
        torch.cuda.synchronize(self.device)  # the copy above ran on torch's stream
        N.rlb_load_state(self.ctx, t)
        self.sync()
        return self

    def macro(self, state: torch.Tensor | None = None, where: str = "device"):
        """(n, eps, beta, ok): n, eps (nz, ny, nx), beta (3, nz, ny, nx); NaN at solid cells;
        ok is False when some cell failed the recovery (outputs are still written)."""
        shp = (self.nz, self.ny, self.nx)
        if where == "device":
            n = torch.empty(shp, dtype=torch.float64, device=self.device)
            e = torch.empty(shp, dtype=torch.float64, device=self.device)
            b = torch.empty((3,) + shp, dtype=torch.float64, device=self.device)
            st = N.rlb_macro(self.ctx, state, n, e, b, N.RLB_DEVICE)
        else:
            n, e, b = np.empty(shp), np.empty(shp), np.empty((3,) + shp)
            st = N.rlb_macro(self.ctx, state, n, e, b, N.RLB_HOST)
        return n, e, b, st == N.RLB_OK

    def stats(self) -> dict:
        return N.rlb_stats(self.ctx)

    def sync(self):
        N.rlb_sync(self.ctx)

    @property
    def launches(self) -> int:
        return N.rlb_launch_count(self.ctx)

    # -- adjoint --------------------------------------------------------------
    def adjoint_macro(self, state, dL_dn, dL_deps, dL_dbeta, lam_out):
        N.rlb_adjoint_macro(self.ctx, state, dL_dn.contiguous(), dL_deps.contiguous(), dL_dbeta.contiguous(), lam_out)

    def adjoint_step(self, state_t, lam_in, lam_out, dtau_acc, dbeta_in_acc):
        N.rlb_adjoint_step(self.ctx, state_t, lam_in, lam_out, dtau_acc, dbeta_in_acc)

    def adjoint_fields(self, n0, eps0, beta0, lam0, dn0, deps0, dbeta0, dbeta_in_acc):
        N.rlb_adjoint_fields(self.ctx, n0, eps0, beta0, lam0, dn0, deps0, dbeta0, dbeta_in_acc)

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            N.rlb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    # -- layout helpers (marshalling between the state layout and arrays) -----
    def state_to_cells(self, state: torch.Tensor) -> torch.Tensor:
        """(38, plane_stride) -> (nz, ny, nx, 2, 19) (cell-major, f then g)."""
        return state[:, :self.N].T.reshape(self.nz, self.ny, self.nx, 2, 19)

    def cells_to_state(self, cells: torch.Tensor) -> torch.Tensor:
        out = torch.zeros((38, self.plane_stride), dtype=self.dtype, device=self.device)
        out[:, :self.N] = cells.reshape(self.N, 38).T.to(self.dtype)
        return out
