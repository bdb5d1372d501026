"""Torch-backed handle around the C ABI: torch supplies device memory and the stream; every step
of the scheme runs in libhweno.so."""
from __future__ import annotations

import contextlib
import ctypes

import numpy as np
import torch

from . import _capi as C

_SYSTEMS = {"advection": C.HWENO_ADVECTION, "burgers": C.HWENO_BURGERS, "euler": C.HWENO_EULER}
_BCS = {"periodic": C.HWENO_BC_PERIODIC, "transmissive": C.HWENO_BC_TRANSMISSIVE,
        "reflective": C.HWENO_BC_REFLECTIVE, "fixed": C.HWENO_BC_FIXED}


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


class Solver:
    """One HWENO-I problem on one GPU.

    state: float64 tensor (nfield, ncomp, ny, nx) on the device, updated in place by step().
    The workspace is a uint8 device tensor of hweno_workspace_bytes() bytes.
    """

    def __init__(self, dim: int, system: str, nx: int, ny: int = 1, dx: float = 1.0, dy: float = None,
                 gamma: float = 1.4, bc: str = "periodic", gamma0: float = None, d0: float = 0.9,
                 eps: float = 1e-10, cfl: float = 0.6, ax: float = 1.0, ay: float = 1.0,
                 device="cuda", stream: torch.cuda.Stream = None, flags: int = 0, grav: float = 0.0,
                 sides=None, fixed=None):
        """flags (HWENO_FLAG_*), grav, sides (four boundary types: x-low, x-high, y-low, y-high) and
        fixed ({side: conserved state}) select the extensions of hweno_create_ex."""
        if not torch.cuda.is_available():
            raise RuntimeError("HWENO solver needs a CUDA device")
        self.lib = C.load()
        self.dim, self.system = int(dim), _SYSTEMS[system] if isinstance(system, str) else int(system)
        self.nx, self.ny = int(nx), (int(ny) if dim == 2 else 1)
        dy = dx if dy is None else dy
        h = ctypes.c_void_p()
        bct = _BCS[bc] if isinstance(bc, str) else int(bc)
        if flags or grav or sides is not None or fixed:
            ext = C.HwenoExt()
            ext.flags = int(flags)
            ext.grav = float(grav)
            for k, t in enumerate(sides if sides is not None else (bct,) * 4):
                ext.side[k] = _BCS[t] if isinstance(t, str) else int(t)
            for k, U in (fixed or {}).items():
                for j, u in enumerate(U):
                    ext.fixed[k][j] = float(u)
            C.check(self.lib.hweno_create_ex(self.dim, self.system, self.nx, self.ny, float(dx), float(dy),
                                             float(gamma), ctypes.byref(ext), ctypes.byref(h)), "hweno_create_ex")
        else:
            C.check(self.lib.hweno_create(self.dim, self.system, self.nx, self.ny, float(dx), float(dy),
                                          float(gamma), bct, ctypes.byref(h)), "hweno_create")
        self.h = h
        if gamma0 is None:
            gamma0 = 0.95 if dim == 1 else 0.99
        C.check(self.lib.hweno_set_params(h, float(gamma0), float(d0), float(eps), float(cfl), float(ax),
                                          float(ay)), "hweno_set_params")
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        C.check(self.lib.hweno_set_stream(h, ctypes.c_void_p(self.stream.cuda_stream)), "hweno_set_stream")
        self.ncomp = (3 if dim == 1 else 4) if self.system == C.HWENO_EULER else 1
        self.nfield = dim + 1
        n = self.lib.hweno_state_doubles(h)
        assert n == self.nfield * self.ncomp * self.nx * self.ny
        # every allocation and fill of the handle's memory is ordered on the handle's stream, the
        # stream its kernels run on (torch's caching allocator ties each block to the stream that
        # allocated it)
        with torch.cuda.stream(self.stream):
            self.state = torch.zeros((self.nfield, self.ncomp, self.ny, self.nx), dtype=torch.float64,
                                     device=self.device)
            self.workspace = torch.empty(int(self.lib.hweno_workspace_bytes(h)), dtype=torch.uint8,
                                         device=self.device)
            C.check(self.lib.hweno_bind(h, _ptr(self.state), _ptr(self.workspace)), "hweno_bind")

    # ------------------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.hweno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @contextlib.contextmanager
    def _ordered(self):
        """Run the body on the handle's stream, ordered after the caller's current stream; on exit
        the caller's stream waits for the handle's.  Tensors appended to the yielded list were
        allocated inside (on the handle's stream) and are handed to the caller: they are marked as
        used on the caller's stream, so the allocator does not hand their memory out again before
        the caller's work on them is done."""
        cur = torch.cuda.current_stream(self.device)
        outs = []
        with torch.cuda.stream(self.stream):
            if self.stream != cur:
                self.stream.wait_stream(cur)
            yield outs
        if self.stream != cur:
            cur.wait_stream(self.stream)
            for t in outs:
                t.record_stream(cur)

    def set_state(self, S) -> None:
        S = torch.as_tensor(np.asarray(S) if not isinstance(S, torch.Tensor) else S, dtype=torch.float64)
        with self._ordered():
            self.state.copy_(S.reshape(self.state.shape).to(self.device, non_blocking=True))

    def rhs(self, S=None):
        """(L(S), M(S)) of one stage as device tensors; S defaults to the bound state.

        S is copied and the outputs are allocated on the handle's stream, which the kernels run on;
        the caller's current stream waits for the kernels before the outputs are handed back."""
        with self._ordered() as outs:
            Sd = self.state if S is None else torch.as_tensor(S, dtype=torch.float64).to(self.device).contiguous()
            Sd = Sd.reshape(self.state.shape)
            L = torch.empty_like(Sd)
            M = torch.empty_like(Sd)
            C.check(self.lib.hweno_rhs(self.h, _ptr(Sd), _ptr(L), _ptr(M)), "hweno_rhs")
            outs += [L, M]
        return L, M

    def step(self, dt: float = 0.0, nsteps: int = 1) -> None:
        with self._ordered():
            C.check(self.lib.hweno_steps(self.h, float(dt), int(nsteps)), "hweno_steps")

    def set_time(self, t: float, t_end: float) -> None:
        C.check(self.lib.hweno_set_time(self.h, float(t), float(t_end)), "hweno_set_time")

    def last_dt(self):
        dt, t = ctypes.c_double(), ctypes.c_double()
        C.check(self.lib.hweno_last_dt(self.h, ctypes.byref(dt), ctypes.byref(t)), "hweno_last_dt")
        return dt.value, t.value

    def max_wavespeed(self):
        ax, ay = ctypes.c_double(), ctypes.c_double()
        C.check(self.lib.hweno_max_wavespeed(self.h, ctypes.byref(ax), ctypes.byref(ay)),
                "hweno_max_wavespeed")
        return ax.value, ay.value

    def sync(self) -> None:
        C.check(self.lib.hweno_sync(self.h), "hweno_sync")

    def upload(self, host: torch.Tensor) -> None:
        """Asynchronous host->device copy of a (pinned) CPU float64 tensor into the state."""
        assert host.dtype == torch.float64 and host.is_contiguous() and host.numel() == self.state.numel()
        C.check(self.lib.hweno_upload(self.h, ctypes.c_void_p(host.data_ptr())), "hweno_upload")

    def download(self, host: torch.Tensor) -> None:
        assert host.dtype == torch.float64 and host.is_contiguous() and host.numel() == self.state.numel()
        C.check(self.lib.hweno_download(self.h, ctypes.c_void_p(host.data_ptr())), "hweno_download")

    def set_profiling(self, on: bool) -> None:
        C.check(self.lib.hweno_set_profiling(self.h, int(bool(on))), "hweno_set_profiling")

    def kernel_times(self):
        """{kind: (total ms, launches)} for kinds cell, face, update since the last query."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_longlong * 3)()
        C.check(self.lib.hweno_kernel_times(self.h, ms, n), "hweno_kernel_times")
        return {k: (ms[i], n[i]) for i, k in enumerate(("cell", "face", "update"))}

    def launch_count(self) -> int:
        return int(self.lib.hweno_launch_count(self.h))

    def pipeline(self, host_in, host_out, nsteps: int = 1, depth: int = 3) -> None:
        """Independent problems of this grid and scheme, host to host (hweno_pipeline): problem i is
        uploaded from the host tensor host_in[i], advanced by nsteps CFL steps and downloaded to
        host_out[i] (float64, contiguous, the state's size; pinned memory lets the copies overlap
        the steps), on `depth` device slots in turn.  Returns when every result is in host memory."""
        n = len(host_in)
        if len(host_out) != n:
            raise ValueError("host_in and host_out differ in length")
        size = self.state.numel()
        for t in list(host_in) + list(host_out):
            if t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != size:
                raise ValueError("pipeline arrays: contiguous float64 host tensors of the state's size")
        need = int(depth) * int(self.lib.hweno_pipeline_slot_bytes(self.h))
        mem = getattr(self, "pipeline_memory", None)
        if mem is None or mem.numel() < need:
            self.pipeline_memory = None
            with torch.cuda.stream(self.stream):
                self.pipeline_memory = torch.empty(need, dtype=torch.uint8, device=self.device)
        ins = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in host_in])
        outs = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in host_out])
        with self._ordered():
            C.check(self.lib.hweno_pipeline(self.h, n, ins, outs, int(nsteps), int(depth),
                                            _ptr(self.pipeline_memory)), "hweno_pipeline")

    # ---- adjoint support (fixed dt and per-stage LF coefficients) ----------------------------
    def _adj_ws(self):
        if getattr(self, "adj_workspace", None) is None:
            self.adj_workspace = torch.empty(int(self.lib.hweno_adjoint_workspace_bytes(self.h)), dtype=torch.uint8,
                                             device=self.device)
        return self.adj_workspace

    def record(self, out7: torch.Tensor) -> None:
        """Copy dt and the three stage alphas of the last step into a device tensor of 7 doubles."""
        with self._ordered():
            C.check(self.lib.hweno_step_record(self.h, ctypes.c_void_p(out7.data_ptr())), "hweno_step_record")

    def step_replay(self, dt: float, alpha6: torch.Tensor) -> None:
        with self._ordered():
            C.check(self.lib.hweno_step_replay(self.h, float(dt), ctypes.c_void_p(alpha6.data_ptr())),
                    "hweno_step_replay")

    def adjoint_step(self, Sn: torch.Tensor, dt: float, alpha6: torch.Tensor, lam_in: torch.Tensor) -> torch.Tensor:
        """(dS^{n+1}/dS^n)^T lam_in for the step from Sn with dt and alpha6 (device tensors)."""
        with self._ordered() as outs:
            ws = self._adj_ws()
            lam_out = torch.empty_like(lam_in)
            C.check(self.lib.hweno_adjoint_step(self.h, ctypes.c_void_p(Sn.data_ptr()), float(dt),
                                                ctypes.c_void_p(alpha6.data_ptr()), ctypes.c_void_p(lam_in.data_ptr()),
                                                ctypes.c_void_p(lam_out.data_ptr()), ctypes.c_void_p(ws.data_ptr())),
                    "hweno_adjoint_step")
            outs.append(lam_out)
        return lam_out

    def step_stages(self, S1: torch.Tensor, S2: torch.Tensor, dt: float = 0.0) -> None:
        """One step (CFL on the device for dt <= 0), copying its stage inputs S1 and S2 out."""
        with self._ordered():
            C.check(self.lib.hweno_step_stages(self.h, float(dt), ctypes.c_void_p(S1.data_ptr()),
                                               ctypes.c_void_p(S2.data_ptr())), "hweno_step_stages")

    def step_replay_stages(self, dt: float, alpha6: torch.Tensor, S1: torch.Tensor, S2: torch.Tensor) -> None:
        """Replay a recorded step, copying its stage inputs S1 and S2 out."""
        with self._ordered():
            C.check(self.lib.hweno_step_replay_stages(self.h, float(dt), ctypes.c_void_p(alpha6.data_ptr()),
                                                      ctypes.c_void_p(S1.data_ptr()), ctypes.c_void_p(S2.data_ptr())),
                    "hweno_step_replay_stages")

    def adjoint_step_stages(self, Sn, S1, S2, dt: float, alpha6: torch.Tensor, lam_in: torch.Tensor) -> torch.Tensor:
        with self._ordered() as outs:
            ws = self._adj_ws()
            lam_out = torch.empty_like(lam_in)
            C.check(self.lib.hweno_adjoint_step_stages(
                self.h, ctypes.c_void_p(Sn.data_ptr()), ctypes.c_void_p(S1.data_ptr()), ctypes.c_void_p(S2.data_ptr()),
                float(dt), ctypes.c_void_p(alpha6.data_ptr()), ctypes.c_void_p(lam_in.data_ptr()),
                ctypes.c_void_p(lam_out.data_ptr()), ctypes.c_void_p(ws.data_ptr())), "hweno_adjoint_step_stages")
            outs.append(lam_out)
        return lam_out

    def run(self, t_end: float, max_steps: int = 10 ** 9) -> int:
        """CFL steps from t = 0 to t_end (last step clamped on the device); returns the step count."""
        n = ctypes.c_int64()
        with self._ordered():
            C.check(self.lib.hweno_run(self.h, float(t_end), int(max_steps), ctypes.byref(n)), "hweno_run")
        return int(n.value)


class Batch:
    """Many independent Euler problems (1D and 2D, uneven sizes) advanced together.

    descs: list of dicts with keys dim, nx, ny (2D), dx, dy (2D), bc ('periodic' or
    'transmissive'), gamma.  The packed device state holds the instances back to back; view(i)
    is instance i's (nfield, ncomp, ny, nx) view.  The batch runs on a stream of its own so that
    its steps can replay a CUDA graph.
    """

    def __init__(self, descs, device="cuda", stream: torch.cuda.Stream = None):
        if not torch.cuda.is_available():
            raise RuntimeError("HWENO batch needs a CUDA device")
        self.lib = C.load()
        self.device = torch.device(device)
        n = len(descs)
        arr = (C.HwenoDesc * n)()
        self.shapes = []
        for i, d in enumerate(descs):
            dim = int(d["dim"])
            nx = int(d["nx"])
            ny = int(d.get("ny", 1)) if dim == 2 else 1
            arr[i] = C.HwenoDesc(dim, C.HWENO_EULER, _BCS[d.get("bc", "periodic")], 0, nx, ny,
                                 float(d["dx"]), float(d.get("dy", d["dx"])), float(d.get("gamma", 1.4)))
            self.shapes.append((dim + 1, 3 if dim == 1 else 4, ny, nx))
        h = ctypes.c_void_p()
        C.check(self.lib.hweno_batch_create(n, arr, ctypes.byref(h)), "hweno_batch_create")
        self.h, self.n = h, n
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        C.check(self.lib.hweno_batch_set_stream(h, ctypes.c_void_p(self.stream.cuda_stream)), "hweno_batch_set_stream")
        total = int(self.lib.hweno_batch_state_doubles(h))
        self.offsets = [int(self.lib.hweno_batch_state_offset(h, i)) for i in range(n)]
        self.state = torch.zeros(total, dtype=torch.float64, device=self.device)
        self.workspace = torch.empty(int(self.lib.hweno_batch_workspace_bytes(h)), dtype=torch.uint8,
                                     device=self.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        C.check(self.lib.hweno_batch_bind(h, ctypes.c_void_p(self.state.data_ptr()),
                                          ctypes.c_void_p(self.workspace.data_ptr())), "hweno_batch_bind")

    def close(self):
        if getattr(self, "h", None):
            self.lib.hweno_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def view(self, i):
        size = int(np.prod(self.shapes[i]))
        return self.state[self.offsets[i]:self.offsets[i] + size].view(self.shapes[i])

    def set_state(self, i, S) -> None:
        S = torch.as_tensor(np.asarray(S) if not isinstance(S, torch.Tensor) else S, dtype=torch.float64)
        with torch.cuda.stream(self.stream):
            self.view(i).copy_(S.reshape(self.shapes[i]).to(self.device, non_blocking=True))

    def set_time(self, t_end: float = 0.0) -> None:
        C.check(self.lib.hweno_batch_set_time(self.h, float(t_end)), "hweno_batch_set_time")

    def step(self, nsteps: int = 1) -> None:
        C.check(self.lib.hweno_batch_step(self.h, int(nsteps)), "hweno_batch_step")

    def step_plain(self, nsteps: int = 1) -> None:
        C.check(self.lib.hweno_batch_step_plain(self.h, int(nsteps)), "hweno_batch_step_plain")

    def dts(self):
        dt = (ctypes.c_double * self.n)()
        t = (ctypes.c_double * self.n)()
        C.check(self.lib.hweno_batch_dts(self.h, dt, t), "hweno_batch_dts")
        return np.array(dt[:]), np.array(t[:])

    def tune(self):
        """Autotune the persistent launch; returns (tiles per item, blocks per SM)."""
        backup = torch.empty_like(self.state)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        tpi, bps = ctypes.c_int(), ctypes.c_int()
        C.check(self.lib.hweno_batch_tune(self.h, ctypes.c_void_p(backup.data_ptr()), ctypes.byref(tpi),
                                          ctypes.byref(bps)), "hweno_batch_tune")
        return tpi.value, bps.value

    def launch_count(self) -> int:
        return int(self.lib.hweno_batch_launch_count(self.h))

    def sync(self) -> None:
        self.stream.synchronize()
