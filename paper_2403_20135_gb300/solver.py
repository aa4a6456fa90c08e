"""Python face of the C ABI: one ``Solver`` per (truncation, grid, nodes, sweeps, dt).

States are torch complex128 CUDA tensors of shape (3, ncoef) holding
(Phi', zeta, div) spectra in the m-major triangular packing of include/sdc.h;
torch provides device memory and the stream, the library does all the work.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import _lib


def _ptr(t: torch.Tensor) -> int:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


class Solver:
    def __init__(self, T: int, nlat: int, nlon: int, nodes: int, sweeps: int, dt: float,
                 radius: float, omega: float, gravity: float, mean_depth: float,
                 precision: int = _lib.SDC_FP64, qdelta_rule: int = _lib.SDC_QDELTA_CLAMPED,
                 method: int = _lib.SDC_METHOD_DSDC, stream: torch.cuda.Stream | None = None):
        self.lib = _lib.load()
        self.T, self.nlat, self.nlon, self.nodes, self.sweeps, self.dt = T, nlat, nlon, nodes, sweeps, dt
        self.phys = _lib.SdcPhys(radius, omega, gravity, mean_depth)
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _lib.check(self.lib.sdc_create(ctypes.byref(h), T, nlat, nlon, nodes, sweeps, dt,
                                       ctypes.byref(self.phys), precision,
                                       ctypes.c_void_p(self.stream.cuda_stream)), "sdc_create")
        self.h = h
        if qdelta_rule != _lib.SDC_QDELTA_CLAMPED:
            self.set_qdelta_rule(qdelta_rule)
        self.ncoef = self.lib.sdc_ncoef(h)
        self.method = _lib.SDC_METHOD_DSDC
        if method != _lib.SDC_METHOD_DSDC:
            self.set_method(method)

    def set_qdelta_rule(self, rule: int):
        """Diagonal q^Delta rule: SDC_QDELTA_CLAMPED, _LITERAL, _MIN_SR_NS, _IMPLICIT_EULER or _MIN_SR_S."""
        _lib.check(self.lib.sdc_set_option(self.h, _lib.SDC_OPT_QDELTA_RULE, rule), "sdc_set_option")

    def set_method(self, method: int):
        """Integrator for step/run: SDC_METHOD_DSDC, SDC_METHOD_SERIAL_SDC or SDC_METHOD_IMEX2."""
        _lib.check(self.lib.sdc_set_option(self.h, _lib.SDC_OPT_METHOD, method), "sdc_set_option")
        self.method = method

    def set_serial_implicit(self, weights: int):
        """Implicit weights of serial IMEX SDC: SDC_SERIAL_IMPLICIT_EULER or SDC_SERIAL_IMPLICIT_LU."""
        _lib.check(self.lib.sdc_set_option(self.h, _lib.SDC_OPT_SERIAL_IMPLICIT, weights), "sdc_set_option")

    def set_legendre(self, source: int):
        """Legendre functions of the FP32 synthesis: SDC_LEGENDRE_TABLE or SDC_LEGENDRE_RECURRENCE."""
        _lib.check(self.lib.sdc_set_option(self.h, _lib.SDC_OPT_LEGENDRE, source), "sdc_set_option")

    def set_chains(self, chains: int):
        """Concurrent state chains of a tendency batch in the step graphs: 1 to 4."""
        _lib.check(self.lib.sdc_set_option(self.h, _lib.SDC_OPT_CHAINS, chains), "sdc_set_option")

    def set_pdl(self, on: int):
        """Programmatic dependent launch in the step graphs: 1 (default) or 0."""
        _lib.check(self.lib.sdc_set_option(self.h, _lib.SDC_OPT_PDL, on), "sdc_set_option")

    @classmethod
    def for_workload(cls, wl, precision: int = _lib.SDC_FP64, **kw):
        import swe_inputs as si
        return cls(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, wl.dt, si.RADIUS, si.OMEGA,
                   si.GRAVITY, si.MEAN_DEPTH, precision=precision, **kw)

    def close(self):
        if getattr(self, "h", None):
            self.lib.sdc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- state helpers -----------------------------------------------------
    def empty_state(self, batch: int | None = None) -> torch.Tensor:
        shape = (3, self.ncoef) if batch is None else (batch, 3, self.ncoef)
        return torch.zeros(shape, dtype=torch.complex128, device="cuda")

    def _check_state(self, t: torch.Tensor, batch: int | None = None):
        want = (3, self.ncoef) if batch is None else (batch, 3, self.ncoef)
        if t.dtype != torch.complex128 or tuple(t.shape) != want:
            raise ValueError(f"state must be complex128 of shape {want}, got {t.dtype} {tuple(t.shape)}")

    # ---- the C ABI ---------------------------------------------------------
    def step(self, state_in: torch.Tensor, state_out: torch.Tensor | None = None, residuals: bool = False):
        self._check_state(state_in)
        if state_out is None:
            state_out = torch.empty_like(state_in)
        self._check_state(state_out)
        res = (ctypes.c_double * (3 * self.sweeps))() if residuals else None
        _lib.check(self.lib.sdc_step(self.h, _ptr(state_in), _ptr(state_out), res), "sdc_step")
        if residuals:
            return state_out, np.array(res[:]).reshape(self.sweeps, 3)
        return state_out

    def save(self, state: torch.Tensor, path: str, step: int = 0) -> None:
        """Write the state and a step index to a checkpoint file (sdc_save)."""
        self._check_state(state)
        _lib.check(self.lib.sdc_save(self.h, _ptr(state), int(step), os.fsencode(path)), "sdc_save")

    def load(self, path: str, state: torch.Tensor | None = None):
        """Read a checkpoint file of this truncation (sdc_load): (state, step)."""
        if state is None:
            state = torch.empty((3, self.ncoef), dtype=torch.complex128, device="cuda")
        self._check_state(state)
        step = ctypes.c_longlong(0)
        _lib.check(self.lib.sdc_load(self.h, _ptr(state), ctypes.byref(step), os.fsencode(path)), "sdc_load")
        return state, step.value

    def run(self, state: torch.Tensor, nsteps: int) -> torch.Tensor:
        self._check_state(state)
        _lib.check(self.lib.sdc_run(self.h, _ptr(state), int(nsteps)), "sdc_run")
        return state

    def tendency(self, states: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        squeeze = states.dim() == 2
        s = states.unsqueeze(0) if squeeze else states
        s = s.contiguous()
        self._check_state(s, s.shape[0])
        o = torch.empty_like(s) if out is None else out
        _lib.check(self.lib.sdc_tendency(self.h, _ptr(s), _ptr(o), s.shape[0]), "sdc_tendency")
        return o[0] if squeeze else o

    # ---- adjoint ---------------------------------------------------------
    def tendency_adjoint(self, states: torch.Tensor, abar: torch.Tensor) -> torch.Tensor:
        """J_E(states)^T abar (batch of states, or one state)."""
        squeeze = states.dim() == 2
        s = (states.unsqueeze(0) if squeeze else states).contiguous()
        a = (abar.unsqueeze(0) if squeeze else abar).contiguous()
        self._check_state(s, s.shape[0])
        self._check_state(a, s.shape[0])
        o = torch.empty_like(s)
        _lib.check(self.lib.sdc_tendency_adjoint(self.h, _ptr(s), _ptr(a), _ptr(o), s.shape[0]),
                   "sdc_tendency_adjoint")
        return o[0] if squeeze else o

    def step_adjoint(self, state: torch.Tensor, ubar_next: torch.Tensor) -> torch.Tensor:
        self._check_state(state)
        self._check_state(ubar_next)
        o = torch.empty_like(state)
        _lib.check(self.lib.sdc_step_adjoint(self.h, _ptr(state), _ptr(ubar_next), _ptr(o)), "sdc_step_adjoint")
        return o

    def run_adjoint(self, state0: torch.Tensor, nsteps: int, ubar_final: torch.Tensor, nsnapshots: int = 8):
        """((d u_N / d u_0)^T ubar_final, number of recomputed forward steps)."""
        self._check_state(state0)
        self._check_state(ubar_final)
        o = torch.empty_like(state0)
        n = ctypes.c_longlong()
        _lib.check(self.lib.sdc_run_adjoint(self.h, _ptr(state0), int(nsteps), int(nsnapshots), _ptr(ubar_final),
                                            _ptr(o), ctypes.byref(n)), "sdc_run_adjoint")
        return o, n.value

    def adjoint_run(self, state0: torch.Tensor, nsteps: int, h_target: torch.Tensor, nsnapshots: int = 8):
        """(loss, gradient) of 0.5 sum (h(T) - h_target)^2 with respect to state0."""
        self._check_state(state0)
        if h_target.dtype != torch.float64 or tuple(h_target.shape) != (self.nlat, self.nlon):
            raise ValueError("h_target must be float64 of shape (nlat, nlon)")
        g = torch.empty_like(state0)
        loss = ctypes.c_double()
        _lib.check(self.lib.sdc_adjoint_run(self.h, _ptr(state0), int(nsteps), int(nsnapshots),
                                            _ptr(h_target.contiguous()), ctypes.byref(loss), _ptr(g)),
                   "sdc_adjoint_run")
        return loss.value, g

    def spec_to_grid(self, spec: torch.Tensor) -> torch.Tensor:
        if spec.dtype != torch.complex128 or tuple(spec.shape) != (self.ncoef,):
            raise ValueError("spec must be complex128 of shape (ncoef,)")
        g = torch.empty((self.nlat, self.nlon), dtype=torch.float64, device="cuda")
        _lib.check(self.lib.sdc_spec_to_grid(self.h, _ptr(spec.contiguous()), _ptr(g)), "sdc_spec_to_grid")
        return g

    def grid_to_spec(self, grid: torch.Tensor) -> torch.Tensor:
        if grid.dtype != torch.float64 or tuple(grid.shape) != (self.nlat, self.nlon):
            raise ValueError("grid must be float64 of shape (nlat, nlon)")
        s = torch.empty(self.ncoef, dtype=torch.complex128, device="cuda")
        _lib.check(self.lib.sdc_grid_to_spec(self.h, _ptr(grid.contiguous()), _ptr(s)), "sdc_grid_to_spec")
        return s

    def grid_coords(self):
        mu = (ctypes.c_double * self.nlat)()
        w = (ctypes.c_double * self.nlat)()
        _lib.check(self.lib.sdc_grid_coords(self.h, mu, w), "sdc_grid_coords")
        return np.array(mu[:]), np.array(w[:])

    def collocation(self):
        tau = (ctypes.c_double * self.nodes)()
        Q = (ctypes.c_double * (self.nodes * self.nodes))()
        _lib.check(self.lib.sdc_collocation(self.h, tau, Q), "sdc_collocation")
        return np.array(tau[:]), np.array(Q[:]).reshape(self.nodes, self.nodes)

    def counters(self):
        a, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _lib.check(self.lib.sdc_counters(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "sdc_counters")
        return a.value, b.value, c.value

    STAGES = ("synthesis", "ring", "analysis", "epilogue", "sweep", "resid")

    def profile_step(self, state: torch.Tensor):
        """One step launched kernel by kernel with CUDA events: {stage: (ms, launches)}."""
        self._check_state(state)
        ms = (ctypes.c_double * 6)()
        nl = (ctypes.c_int * 6)()
        _lib.check(self.lib.sdc_profile_step(self.h, _ptr(state), ms, nl), "sdc_profile_step")
        return {k: (ms[i], nl[i]) for i, k in enumerate(self.STAGES)}

    def sync(self):
        """Wait for the stream; raises if a kernel reported an expired wait."""
        _lib.check(self.lib.sdc_sync(self.h), "sdc_sync")

    def launches_per_step(self) -> int:
        n = ctypes.c_int()
        _lib.check(self.lib.sdc_launches_per_step(self.h, ctypes.byref(n)), "sdc_launches_per_step")
        return n.value

    # ---- initial states ----------------------------------------------------
    def initial_state(self, wl) -> torch.Tensor:
        """Seeded workload state: zeta/div spectra from the input law, Phi' from the
        height bumps on this solver's Gauss grid analysed by the library."""
        import swe_inputs as si
        zeta, div = si.vorticity_divergence(wl)
        mu, _ = self.grid_coords()
        lam = 2.0 * np.pi * np.arange(self.nlon) / self.nlon
        hb = si.bump_height(wl, mu, lam, radius=self.phys.radius)
        grid = torch.from_numpy(self.phys.gravity * hb).to("cuda")
        u = self.empty_state()
        u[0] = self.grid_to_spec(grid)
        u[1] = torch.from_numpy(zeta).to("cuda")
        u[2] = torch.from_numpy(div).to("cuda")
        return u


def fp64_fma_rate(iters: int = 4096, repeats: int = 5) -> float:
    """Measured FP64 FMA rate of the current device in TFLOP/s (sdc_fp64_fma_rate)."""
    lib = _lib.load()
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = ctypes.c_double()
    stream = torch.cuda.current_stream().cuda_stream
    _lib.check(lib.sdc_fp64_fma_rate(iters, repeats, stream, _ptr(sink), ctypes.byref(out)), "sdc_fp64_fma_rate")
    return out.value
