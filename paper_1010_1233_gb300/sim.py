"""Python front end of libflb: a context over one or more replicas.

PyTorch provides the device workspace and the CUDA stream; every step of the
method runs in the library's kernels through the C ABI.
"""
import ctypes

import numpy as np
import torch

from . import _lib as L

_NONCONSERVED = {"D2Q9": (3, 4, 5, 6, 7, 8), "D1Q3": (2,), "D3Q15": tuple(range(4, 15)),
                 "D3Q19": tuple(range(4, 19))}
_LATTICE = {"D2Q9": L.FLB_D2Q9, "D1Q3": L.FLB_D1Q3, "D3Q15": L.FLB_D3Q15, "D3Q19": L.FLB_D3Q19}
_Q = {"D1Q3": 3, "D2Q9": 9, "D3Q15": 15, "D3Q19": 19}
_3D = ("D3Q15", "D3Q19")
_PREC = {"fp64": L.FLB_FP64, "fp32": L.FLB_FP32_DEV}


def replica_struct(p):
    """flb_replica from a parameter dict (paper_1010_1233_gb300.workloads.replica)."""
    s = L.flb_replica()
    s.lattice = _LATTICE[p["lattice"]]
    s.nx = int(p["nx"])
    s.ny = int(p["ny"]) if p["lattice"] != "D1Q3" else 1
    s.nz = int(p.get("nz", 1)) if p["lattice"] in _3D else 1
    tau = list(p["tau"]) + [1.0] * (20 - len(p["tau"]))
    for a in range(20):
        s.tau[a] = float(tau[a])
    s.rho0 = float(p["rho0"])
    s.kT = float(p["kT"])
    u0 = list(p["u0"]) + [0.0] * (3 - len(p["u0"]))
    s.u0[0], s.u0[1], s.u0[2] = float(u0[0]), float(u0[1]), float(u0[2])
    s.seed = int(p["seed"]) & 0xFFFFFFFFFFFFFFFF
    s.stream = int(p.get("stream", 0))
    nm = p.get("noise_mask")
    s.noise_mask = sum(1 << a for a in _NONCONSERVED[p["lattice"]]) if nm is None else int(nm)
    s.init_mode = int(p.get("init_mode", 0))
    s.field_mask = sum(1 << f for f in p.get("fields", ()))
    s.noise_mode = int(p.get("noise_mode", 0))
    return s


def stability(p, max_k=64):
    """(spectral radius, (jx, jy, jz)) of the linearised one-step operator of replica
    parameters p over a k-grid (flb_stability); a radius above 1 means the run diverges."""
    s = replica_struct(p)
    r = ctypes.c_double()
    k = (ctypes.c_int32 * 3)()
    L.check(L.lib().flb_stability(ctypes.byref(s), int(max_k), ctypes.byref(r), k))
    return float(r.value), (int(k[0]), int(k[1]), int(k[2]))


def bf16_bits(x):
    """bfloat16 bit patterns (round to nearest even) of an FP32 array, via torch."""
    t = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16)


class Sim:
    """A batch of replicas sharing one lattice type and storage precision."""

    def __init__(self, replicas, precision="fp32", device=None, stream=None):
        if isinstance(replicas, dict):
            replicas = [replicas]
        self.params = [dict(p) for p in replicas]
        self.precision = precision
        n = len(self.params)
        arr = (L.flb_replica * n)(*[replica_struct(p) for p in self.params])
        self._reps = arr
        lib = L.lib()
        nbytes = ctypes.c_size_t()
        L.check(lib.flb_workspace_bytes(_PREC[precision], arr, n, ctypes.byref(nbytes)))
        self.device = torch.device(device or "cuda")
        self.workspace = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8, device=self.device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self._tc = None                      # time-correlator buffer (set_time_correlator)
        ctx = ctypes.c_void_p()
        L.check(lib.flb_create(_PREC[precision], arr, n, ctypes.c_void_p(self.workspace.data_ptr()),
                               self.workspace.numel(), ctypes.c_void_p(self.stream.cuda_stream),
                               ctypes.byref(ctx)))
        self._ctx = ctx
        self.workspace_bytes = int(nbytes.value)

    # -- stepping ---------------------------------------------------------
    def run(self, n_steps, sample_every=0):
        L.check(L.lib().flb_run(self._ctx, int(n_steps), int(sample_every)))
        return self

    def sync(self):
        L.check(L.lib().flb_sync(self._ctx))

    def reset_stats(self):
        L.check(L.lib().flb_reset_stats(self._ctx))

    @property
    def step(self):
        v = ctypes.c_uint64()
        L.check(L.lib().flb_get_step(self._ctx, ctypes.byref(v)))
        return int(v.value)

    # -- results ----------------------------------------------------------
    def _shape(self, r):
        if not 0 <= r < len(self.params):
            raise L.FlbError(L.FLB_EINVAL, f"replica {r} out of range")
        p = self.params[r]
        return (p["ny"] if p["lattice"] == "D2Q9" else 1, p["nx"])

    def _dims(self, r):
        """Lattice shape of replica r: (nz, ny, nx) for D3Q15 / D3Q19, else (ny, nx)."""
        p = self.params[r] if 0 <= r < len(self.params) else None
        if p is not None and p["lattice"] in _3D:
            return (int(p["nz"]), int(p["ny"]), int(p["nx"]))
        return self._shape(r)

    def correlator(self, r, a, b, with_count=False):
        ny, nx = self._shape(r)
        out = np.empty(ny * nx * 2)
        n = ctypes.c_uint64()
        L.check(L.lib().flb_get_correlator(self._ctx, r, a, b,
                                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(n)))
        c = out[0::2] + 1j * out[1::2]
        c = c.reshape(ny, nx)
        return (c, int(n.value)) if with_count else c

    def populations(self, r=0):
        dims = self._dims(r)
        q = _Q[self.params[r]["lattice"]]
        out = np.empty((q,) + dims)
        L.check(L.lib().flb_get_populations(self._ctx, r, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def populations_window(self, x0, y0, w, h, r=0):
        """Populations [q][h][w] of the window starting at (x0, y0) (inside the lattice)."""
        self._shape(r)
        q = 9 if self.params[r]["lattice"] == "D2Q9" else 3
        out = np.empty((q, h, w))
        L.check(L.lib().flb_get_populations_window(self._ctx, r, x0, y0, w, h,
                                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def fields(self, r=0):
        """Fields of the most recent sample, [n_fields] + lattice shape, in increasing field id order."""
        dims = self._dims(r)
        F = len(self.params[r].get("fields", ()))
        out = np.empty((F,) + dims)
        L.check(L.lib().flb_get_fields(self._ctx, r, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def set_populations(self, f, r=0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        L.check(L.lib().flb_set_populations(self._ctx, r, f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def conserved(self, r=0):
        """Lattice sums (rho, j_x, j_y) (3D lattices: (rho, j_x, j_y, j_z)) of the stored state."""
        out = np.empty(4)
        L.check(L.lib().flb_get_conserved(self._ctx, r, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out if self.params[min(max(r, 0), len(self.params) - 1)]["lattice"] in _3D else out[:3]

    # -- learned noise scale ----------------------------------------------
    def set_mlp(self, weights=None):
        """weights: dict W1 (32,3), b1, W2 (32,32), b2, W3 (6,32), b3 (FP32); None disables."""
        lib = L.lib()
        if weights is None:
            L.check(lib.flb_set_mlp(self._ctx, None, None, 0))
            return
        w = np.concatenate([bf16_bits(weights[k]).ravel() for k in ("W1", "W2", "W3")])
        b = np.concatenate([np.asarray(weights[k], np.float32).ravel() for k in ("b1", "b2", "b3")])
        w = np.ascontiguousarray(w, dtype=np.uint16)
        b = np.ascontiguousarray(b, dtype=np.float32)
        L.check(lib.flb_set_mlp(self._ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)),
                                b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 1))

    # -- time correlators -------------------------------------------------
    def set_time_correlator(self, kpoints, n_lags):
        """Accumulate F_ab(k, tau) at the wave vectors kpoints = [(ky, kx), ...] (3D lattices:
        [(kz, ky, kx), ...]) for lags 0..n_lags-1 (samples); n_lags = 0 switches them off."""
        lib = L.lib()
        if n_lags == 0:
            L.check(lib.flb_set_time_correlator(self._ctx, 0, 0, None, None, None, 0))
            self._tc = None
            return
        kp = [tuple(int(v) for v in k) for k in kpoints]
        kp = [k if len(k) == 3 else (0,) + k for k in kp]
        kz = np.ascontiguousarray([k[0] for k in kp], dtype=np.int32)
        ky = np.ascontiguousarray([k[1] for k in kp], dtype=np.int32)
        kx = np.ascontiguousarray([k[2] for k in kp], dtype=np.int32)
        n = ctypes.c_size_t()
        L.check(lib.flb_time_correlator_bytes(self._ctx, int(n_lags), len(kx), ctypes.byref(n)))
        buf = torch.empty(int(n.value) + 256, dtype=torch.uint8, device=self.device)
        off = (-buf.data_ptr()) % 256
        L.check(lib.flb_set_time_correlator3(self._ctx, int(n_lags), len(kx), kx.ctypes.data, ky.ctypes.data,
                                             kz.ctypes.data, ctypes.c_void_p(buf.data_ptr() + off), int(n.value)))
        self._tc = (buf, int(n_lags), len(kx))

    def time_correlator(self, r, a, b, with_count=False):
        """Normalised F_ab(k, tau) of replica r, complex (n_lags, n_k)."""
        _, T, nk = self._tc
        out = np.empty(2 * T * nk)
        cnt = ctypes.c_uint64()
        L.check(L.lib().flb_get_time_correlator(self._ctx, int(r), int(a), int(b),
                                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                ctypes.byref(cnt)))
        v = out[0::2].reshape(T, nk) + 1j * out[1::2].reshape(T, nk)
        return (v, int(cnt.value)) if with_count else v

    # -- launch configuration ---------------------------------------------
    def set_step_config(self, vec, grid_blocks=0, staged=0):
        L.check(L.lib().flb_set_step_config(self._ctx, int(vec), int(grid_blocks), int(staged)))

    def step_config(self):
        """(vec, grid blocks, staged) of the step kernel."""
        v, g, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.check(L.lib().flb_get_step_config(self._ctx, ctypes.byref(v), ctypes.byref(g), ctypes.byref(s)))
        return int(v.value), int(g.value), int(s.value)

    def set_network_engine(self, engine):
        """'warp' (warp-level MMAs, default) or 'tcgen05' (tensor-memory MMAs)."""
        e = {"warp": L.FLB_NET_WARP, "tcgen05": L.FLB_NET_TCGEN05}[engine] if isinstance(engine, str) else int(engine)
        L.check(L.lib().flb_set_network_engine(self._ctx, e))

    def network_engine(self):
        e = ctypes.c_int()
        L.check(L.lib().flb_get_network_engine(self._ctx, ctypes.byref(e)))
        return "tcgen05" if e.value == L.FLB_NET_TCGEN05 else "warp"

    def kernel_launches(self):
        """Kernels flb_run has issued on this context (replayed graphs count their kernels)."""
        n = ctypes.c_uint64()
        L.check(L.lib().flb_kernel_launches(self._ctx, ctypes.byref(n)))
        return int(n.value)

    def set_graphs(self, enable=True):
        L.check(L.lib().flb_set_graphs(self._ctx, int(bool(enable))))

    def probe_wait_timeout(self, limit_clocks):
        """Failure-detection check: one bounded device wait that nothing completes; the
        next sync() raises FlbError(FLB_ETIMEOUT) and the status stays set."""
        L.check(L.lib().flb_probe_wait_timeout(self._ctx, int(limit_clocks)))

    def autotune(self, trials=5):
        """Pick the fastest step-kernel configuration; returns (vec, grid, staged, ms per step)."""
        v, g, s, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        L.check(L.lib().flb_autotune(self._ctx, int(trials), ctypes.byref(v), ctypes.byref(g), ctypes.byref(s),
                                     ctypes.byref(ms)))
        return int(v.value), int(g.value), int(s.value), float(ms.value)

    # -- checkpoint -------------------------------------------------------
    def save(self):
        lib = L.lib()
        n = ctypes.c_size_t()
        L.check(lib.flb_save(self._ctx, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        L.check(lib.flb_save(self._ctx, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def load(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        L.check(L.lib().flb_load(self._ctx, buf, len(blob)))

    def close(self):
        if getattr(self, "_ctx", None):
            L.lib().flb_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def philox(sites, step, call, tag, stream, seed, fp32=False, device="cuda"):
    """Philox words (n, 4) and normals (n, 4) exactly as the step kernels draw them."""
    s = torch.as_tensor(np.asarray(sites, dtype=np.uint32).view(np.int32), device=device)
    n = s.numel()
    words = torch.empty(4 * n, dtype=torch.int32, device=device)
    normals = torch.empty(4 * n, dtype=torch.float64, device=device)
    st = torch.cuda.current_stream()
    L.check(L.lib().flb_philox(ctypes.c_void_p(s.data_ptr()), n, step, call, tag, stream, seed, int(fp32),
                               ctypes.c_void_p(words.data_ptr()), ctypes.c_void_p(normals.data_ptr()),
                               ctypes.c_void_p(st.cuda_stream)))
    torch.cuda.synchronize()
    return (words.cpu().numpy().view(np.uint32).reshape(n, 4), normals.cpu().numpy().reshape(n, 4))


def spectra_sizes(F, ny, nx, precision="fp32"):
    """(scratch bytes, number of FP64 pair sums) of flb_spectra_accumulate."""
    b, n = ctypes.c_size_t(), ctypes.c_size_t()
    L.check(L.lib().flb_spectra_scratch_bytes(_PREC[precision], nx, ny, F, ctypes.byref(b), ctypes.byref(n)))
    return int(b.value), int(n.value)


def spectra_accumulate(fields, sums=None, mean0=None, scratch=None):
    """Add X_a(k) X_b(k)^* of every pair of the device fields (F, ny, nx) to FP64 sums.

    fields: CUDA tensor, float32 (FP32 transforms) or float64.  Returns (sums, mean0),
    allocating zeroed ones when not given.  The pair layout is that of flb.h.
    """
    F, ny, nx = fields.shape
    precision = "fp64" if fields.dtype == torch.float64 else "fp32"
    nb, ns = spectra_sizes(F, ny, nx, precision)
    dev = fields.device
    if sums is None:
        sums = torch.zeros(ns, dtype=torch.float64, device=dev)
    if mean0 is None:
        mean0 = torch.zeros(F, dtype=torch.float64, device=dev)
    if scratch is None:
        scratch = torch.empty(nb, dtype=torch.uint8, device=dev)
    fields = fields.contiguous()
    st = torch.cuda.current_stream(dev)
    L.check(L.lib().flb_spectra_accumulate(_PREC[precision], nx, ny, F, ctypes.c_void_p(fields.data_ptr()),
                                           ctypes.c_void_p(sums.data_ptr()), ctypes.c_void_p(mean0.data_ptr()),
                                           ctypes.c_void_p(scratch.data_ptr()), scratch.numel(),
                                           ctypes.c_void_p(st.cuda_stream)))
    return sums, mean0


def unpack_pair_sums(sums, F, ny, nx):
    """Split the flat pair-sum array into {(a, b): complex (ny, nx/2+1)} (host numpy)."""
    s = sums.detach().cpu().numpy() if hasattr(sums, "detach") else np.asarray(sums)
    hn = nx // 2 + 1
    out, off = {}, 0
    for a in range(F):
        for b in range(a, F):
            n = ny * hn
            if a == b:
                out[(a, b)] = s[off:off + n].reshape(ny, hn).astype(np.complex128)
                off += n
            else:
                v = s[off:off + 2 * n].reshape(ny, hn, 2)
                out[(a, b)] = v[..., 0] + 1j * v[..., 1]
                off += 2 * n
    return out
