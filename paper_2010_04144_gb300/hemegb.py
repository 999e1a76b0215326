"""Python binding of the C ABI in include/hemegb.h (libhemegb.so).

Argument marshalling only: every step of the hot path runs in the library's
sm_103a kernels.  PyTorch supplies device memory (through the allocator hook)
and the CUDA stream; nothing here computes lattice-Boltzmann arithmetic.

The module-level ``hg_*`` functions keep the C names; ``Context`` and
``Domain`` wrap them for convenience.  Loading fails loudly if the extension
has not been built (``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhemegb.so")

HG_OK, HG_ERR_ARG, HG_ERR_OOM, HG_ERR_CUDA, HG_ERR_TIMEOUT, HG_ERR_STATE = 0, -1, -2, -3, -4, -5
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
SCHEME = {"ab": 0, "aa": 1}
COUPLE = {"forward": 0, "alternate": 1}
ORDER = {"morton": 0, "rows": 1, "bricks": 2}
EXCHANGE = {"direct": 0, "staged": 1}
FAULT_ALLOC, FAULT_DEVICE_WAIT = 1, 2
STORE_DTYPE = {0: np.float32, 1: np.float16, 2: None}  # bf16 is returned as uint16 bits


class HgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hemegb error {code}: {msg}")
        self.code = code


class hg_iolet(C.Structure):
    _fields_ = [("kind", C.c_int32), ("profile", C.c_int32), ("pulse", C.c_int32),
                ("reserved", C.c_int32), ("value", C.c_double), ("period", C.c_double),
                ("centre", C.c_int64 * 3), ("axis", C.c_int64 * 3), ("radius", C.c_int64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class hg_ctx_params(C.Structure):
    _fields_ = [("device", C.c_int32), ("storage", C.c_int32), ("scheme", C.c_int32),
                ("block_size", C.c_int32), ("sites_per_thread", C.c_int32),
                ("graph_steps", C.c_int32), ("kernel_variant", C.c_int32),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class hg_lb_params(C.Structure):
    _fields_ = [("tau", C.c_double), ("ordering", C.c_int32), ("reserved", C.c_int32)]


class hg_split_params(C.Structure):
    _fields_ = [("n_parts", C.c_int32), ("exchange", C.c_int32), ("boundary_weight", C.c_double)]


class hg_pair(C.Structure):
    _fields_ = [("src_iolet", C.c_int32), ("dst_iolet", C.c_int32), ("factor", C.c_double)]


_lib = None

_SIGS = {
    "hg_ctx_create": ([C.POINTER(hg_ctx_params), C.POINTER(C.c_void_p)], C.c_int),
    "hg_ctx_destroy": ([C.c_void_p], C.c_int),
    "hg_last_error": ([C.c_void_p], C.c_char_p),
    "hg_sync": ([C.c_void_p], C.c_int),
    "hg_domain_create": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                          C.POINTER(hg_lb_params), C.POINTER(C.c_void_p)], C.c_int),
    "hg_domain_destroy": ([C.c_void_p], C.c_int),
    "hg_domain_info": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
                       C.c_int),
    "hg_domain_runs": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_encode_runs": ([C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                        C.c_void_p, C.c_void_p], C.c_int),
    "hg_domain_sites": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_domain_neighbours": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_couple": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32], C.c_int),
    "hg_set_coupling_mode": ([C.c_void_p, C.c_int32], C.c_int),
    "hg_build_neighbours": ([C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "hg_coupling_factors": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hg_step": ([C.c_void_p, C.c_int64], C.c_int),
    "hg_step_domains": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_int64], C.c_int),
    "hg_step_profiled": ([C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hg_read_macroscopic": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hg_read_macroscopic_device": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_read_iolet_stats": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_read_boundary_values": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_read_iolet_forces": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_mass": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_state_bytes": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_save_state": ([C.c_void_p, C.c_void_p, C.c_int64], C.c_int),
    "hg_load_state": ([C.c_void_p, C.c_void_p, C.c_int64], C.c_int),
    "hg_read_state": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_ctx_set_launch": ([C.c_void_p, C.c_int32, C.c_int32, C.c_int32], C.c_int),
    "hg_mass_noalloc": ([C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p],
                        C.c_int),
    "hg_state_check": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hg_read_adjacent_moments": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hg_ctx_inject_fault": ([C.c_void_p, C.c_int32, C.c_int64], C.c_int),
    "hg_split_layout": ([C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                         C.c_void_p], C.c_int),
    "hg_split_create": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.POINTER(hg_lb_params),
                         C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "hg_split_destroy": ([C.c_void_p], C.c_int),
    "hg_split_info": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "hg_split_step": ([C.c_void_p, C.c_int64], C.c_int),
    "hg_split_read_macroscopic": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_split_read_state": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_split_read_iolet_stats": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_split_read_boundary_values": ([C.c_void_p, C.c_void_p], C.c_int),
    "hg_split_mass": ([C.c_void_p, C.c_void_p], C.c_int),
}


def lib():
    """Load libhemegb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"hemegb CUDA extension missing ({LIB_PATH}); "
                               "run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None and a.size else None


def _check(rc, ctx_handle=None):
    if rc != HG_OK:
        msg = lib().hg_last_error(ctx_handle).decode() if ctx_handle else ""
        raise HgError(rc, msg)


def iolet_struct_array(iolets):
    arr = (hg_iolet * max(1, len(iolets)))()
    for k, d in enumerate(iolets):
        e = arr[k]
        e.kind, e.profile, e.pulse = int(d.kind), int(d.profile), int(d.pulse)
        e.value, e.period = float(d.value), float(d.period)
        for j in range(3):
            e.centre[j] = int(d.centre[j])
            e.axis[j] = int(d.axis[j])
        e.radius = int(d.radius)
    return arr


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, kept alive while the library holds it."""

    def __init__(self, device):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        self.live = {}
        self.c_alloc = ALLOC_FN(self._alloc)
        self.c_free = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:  # out of memory: report NULL, the library returns HG_ERR_OOM
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, nbytes, user):
        self.live.pop(int(ptr), None)


def build_neighbours(xyz, iolets):
    """Host-only canonical order and neighbour table (what a domain build computes):
    returns (xyz_canonical (n, 3) int32, nbr (18, n) int32)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    n = xyz.shape[0]
    arr = iolet_struct_array(iolets)
    xs = np.zeros((max(1, n), 3), np.int32)
    nbr = np.zeros((18, max(1, n)), np.int32)
    _check(lib().hg_build_neighbours(_p(xyz), n, arr, len(iolets), _p(xs), _p(nbr)))
    return xs[:n], nbr[:, :n]


def encode_runs(nbr, n=None, n_ref=None, scheme="ab"):
    """Host-only run encoding (hg_encode_runs) of a device neighbour table nbr
    (18, row_stride) int32 for sites [0, n) (default: every column), fluid entries in
    [0, n_ref) (default n): returns (lword (row_stride,) uint32, run0 (chunks,) int32,
    rdelta (n_runs, 18) int32), or None when the table does not compress."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    stride = nbr.shape[1]
    n = stride if n is None else int(n)
    n_ref = n if n_ref is None else int(n_ref)
    lword = np.zeros(stride, np.uint32)
    run0 = np.zeros((stride + 1023) // 1024, np.int32)
    rdelta = np.zeros((n * 16 // 72 + 1, 18), np.int32)
    nr = C.c_int64()
    sch = SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
    _check(lib().hg_encode_runs(_p(nbr), n, n_ref, stride, sch, _p(lword), _p(run0), _p(rdelta), C.byref(nr)))
    if nr.value == 0:
        return None
    return lword, run0, rdelta[:nr.value]


def split_layout(xyz, iolets, n_parts, boundary_weight=1.0):
    """Host-only partition of a domain (Section 2.2 / 2.2.1): (first (k+1,), ghosts (k,),
    halo (k, k) with halo[q, p] = values partition p pulls from partition q per step)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    sp = hg_split_params(int(n_parts), 0, float(boundary_weight))
    first = np.zeros(n_parts + 1, np.int64)
    ghosts = np.zeros(n_parts, np.int64)
    halo = np.zeros((n_parts, n_parts), np.int64)
    _check(lib().hg_split_layout(_p(xyz), xyz.shape[0], iolet_struct_array(iolets), len(iolets), C.byref(sp),
                                 _p(first), _p(ghosts), _p(halo)))
    return first, ghosts, halo


def hg_coupling_factors(art_centres, art_areas, ven_centres, ven_areas, uniforms):
    """Section 3 coupling map + factors: returns (assign, dist, dp, factor) numpy arrays."""
    ac = np.ascontiguousarray(art_centres, dtype=np.int64).reshape(-1, 3)
    vc = np.ascontiguousarray(ven_centres, dtype=np.int64).reshape(-1, 3)
    aa = np.ascontiguousarray(art_areas, dtype=np.float64)
    va = np.ascontiguousarray(ven_areas, dtype=np.float64)
    un = np.ascontiguousarray(uniforms, dtype=np.float64)
    nv = vc.shape[0]
    assign = np.zeros(nv, np.int32)
    dist, dp, fac = (np.zeros(nv, np.float64) for _ in range(3))
    rc = lib().hg_coupling_factors(_p(ac), _p(aa), ac.shape[0], _p(vc), _p(va), nv, _p(un),
                                   _p(assign), _p(dist), _p(dp), _p(fac))
    _check(rc)
    return assign, dist, dp, fac


class Context:
    """One device, one stream, one storage type and propagation scheme."""

    def __init__(self, device=0, storage="f32", scheme="ab", block_size=0, sites_per_thread=0,
                 graph_steps=0, stream=None, torch_memory=True, kernel_variant=0):
        import torch

        self.torch = torch
        self.device = device
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.scheme = SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
        torch.cuda.set_device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        p = hg_ctx_params()
        p.device, p.storage, p.scheme = device, self.storage, self.scheme
        p.block_size, p.sites_per_thread, p.graph_steps = block_size, sites_per_thread, graph_steps
        p.kernel_variant = kernel_variant
        p.stream = self.stream.cuda_stream
        self._alloc = _TorchAllocator(device) if torch_memory else None
        if self._alloc is not None:
            p.alloc, p.free = self._alloc.c_alloc, self._alloc.c_free
        h = C.c_void_p()
        _check(lib().hg_ctx_create(C.byref(p), C.byref(h)))
        self.h = h
        self.launch = (int(block_size), int(sites_per_thread), int(kernel_variant))
        self.domains = []

    def _ck(self, rc):
        _check(rc, self.h)

    def domain(self, xyz, iolets, tau=0.8, ordering="morton"):
        return Domain(self, xyz, iolets, tau, ordering)

    def split(self, xyz, iolets, n_parts, tau=0.8, boundary_weight=1.0, ordering="morton", exchange="direct"):
        return Split(self, xyz, iolets, n_parts, tau, boundary_weight, ordering, exchange)

    def inject_fault(self, kind, arg=0):
        """Host-side fault injection (FAULT_ALLOC: the arg-th next allocation fails;
        FAULT_DEVICE_WAIT: the device error word is set, hg_sync then reports a timeout)."""
        self._ck(lib().hg_ctx_inject_fault(self.h, int(kind), int(arg)))

    def couple(self, src, dst, pairs):
        arr = (hg_pair * max(1, len(pairs)))()
        for j, (sk, dk, f) in enumerate(pairs):
            arr[j].src_iolet, arr[j].dst_iolet, arr[j].factor = int(sk), int(dk), float(f)
        self._ck(lib().hg_couple(self.h, src.h, dst.h, arr, len(pairs)))

    def set_coupling_mode(self, mode):
        """"forward" (every step) or "alternate" (forward / reverse exchanges, Section 3)."""
        m = COUPLE[mode] if isinstance(mode, str) else int(mode)
        self._ck(lib().hg_set_coupling_mode(self.h, m))

    def set_launch(self, block_size, sites_per_thread, kernel_variant=0):
        self._ck(lib().hg_ctx_set_launch(self.h, int(block_size), int(sites_per_thread),
                                         int(kernel_variant)))
        self.launch = (int(block_size), int(sites_per_thread), int(kernel_variant))

    def step(self, n):
        self._ck(lib().hg_step(self.h, int(n)))

    def step_domains(self, doms, n):
        arr = (C.c_void_p * max(1, len(doms)))(*[d.h for d in doms])
        self._ck(lib().hg_step_domains(self.h, arr, len(doms), int(n)))

    def step_profiled(self, n, per_step=False):
        """Run n steps with CUDA events around every kernel: (stream-collide ms, iolet ms)
        totals, plus the (n, 2) per-step array when per_step is true."""
        a, b = C.c_double(), C.c_double()
        arr = np.zeros((max(1, int(n)), 2), np.float32)
        self._ck(lib().hg_step_profiled(self.h, int(n), C.byref(a), C.byref(b), _p(arr)))
        if per_step:
            return a.value, b.value, arr[: int(n)]
        return a.value, b.value

    def sync(self):
        self._ck(lib().hg_sync(self.h))

    def close(self):
        if self.h:
            lib().hg_ctx_destroy(self.h)
            self.h = None
            for d in self.domains:
                d.h = None
            self.domains = []
            for sp in getattr(self, "splits", []):
                sp.h = None
            self.splits = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Domain:
    def __init__(self, ctx: Context, xyz, iolets, tau=0.8, ordering="morton"):
        self.ctx = ctx
        xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
        self._io = iolet_struct_array(iolets)
        lb = hg_lb_params()
        lb.tau = float(tau)
        lb.ordering = ORDER[ordering] if isinstance(ordering, str) else int(ordering)
        self.ordering = lb.ordering
        h = C.c_void_p()
        ctx._ck(lib().hg_domain_create(ctx.h, _p(xyz), xyz.shape[0], self._io, len(iolets),
                                       C.byref(lb), C.byref(h)))
        self.h = h
        self.n_iolets = len(iolets)
        ctx.domains.append(self)
        self.n = self.info()["n_sites"]

    def info(self):
        n, nio, nadj, step, nb = (C.c_int64(), C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64())
        self.ctx._ck(lib().hg_domain_info(self.h, C.byref(n), C.byref(nio), C.byref(nadj),
                                          C.byref(step), C.byref(nb)))
        runs = C.c_int64()
        self.ctx._ck(lib().hg_domain_runs(self.h, C.byref(runs)))
        return dict(n_sites=n.value, n_iolets=nio.value, n_adjacent=nadj.value, step=step.value,
                    device_bytes=nb.value, n_runs=runs.value)

    @property
    def step(self):
        return self.info()["step"]

    def sites(self):
        out = np.zeros((self.n, 3), np.int32)
        self.ctx._ck(lib().hg_domain_sites(self.h, _p(out)))
        return out

    def neighbours(self):
        out = np.zeros((18, self.n), np.int32)
        self.ctx._ck(lib().hg_domain_neighbours(self.h, _p(out)))
        return out

    def macroscopic(self):
        out = np.zeros((self.n, 4), np.float32)
        st = C.c_int64()
        self.ctx._ck(lib().hg_read_macroscopic(self.h, _p(out), C.byref(st)))
        return out

    def macroscopic_into(self, tensor):
        """Write (drho, ux, uy, uz) into a CUDA float32 tensor of shape (n, 4), asynchronously."""
        assert tensor.is_cuda and tensor.dtype == self.ctx.torch.float32 and tensor.is_contiguous()
        assert tuple(tensor.shape) == (self.n, 4)
        self.ctx._ck(lib().hg_read_macroscopic_device(self.h, C.c_void_p(tensor.data_ptr())))

    def iolet_stats(self):
        out = np.zeros((max(1, self.n_iolets), 3), np.float64)
        self.ctx._ck(lib().hg_read_iolet_stats(self.h, _p(out)))
        return out[: self.n_iolets]

    def boundary_values(self):
        out = np.zeros(max(1, self.n_iolets), np.float32)
        self.ctx._ck(lib().hg_read_boundary_values(self.h, _p(out)))
        return out[: self.n_iolets]

    def iolet_forces(self):
        """Body-force density per iolet for the next step, (n_iolets, 3) float32."""
        out = np.zeros((max(1, self.n_iolets), 3), np.float32)
        self.ctx._ck(lib().hg_read_iolet_forces(self.h, _p(out)))
        return out[: self.n_iolets]

    def mass(self):
        out = C.c_double()
        self.ctx._ck(lib().hg_mass(self.h, C.byref(out)))
        return out.value

    def state_check(self):
        """(mass, number of non-finite stored values, return code) -- HG_ERR_STATE when
        the state holds a NaN or an Inf."""
        m, bad = C.c_double(), C.c_int64()
        rc = lib().hg_state_check(self.h, C.byref(m), C.byref(bad))
        if rc not in (HG_OK, HG_ERR_STATE):
            self.ctx._ck(rc)
        return m.value, bad.value, rc

    def adjacent_moments(self):
        """Sites next to any iolet (canonical order) and the FP32 moments (drho, ux, uy, uz)
        the last step's iolet means were taken over: (sites (m,) int64, moments (m, 4))."""
        m = self.info()["n_adjacent"]
        sites = np.zeros(max(1, m), np.int64)
        mom = np.zeros((max(1, m), 4), np.float32)
        self.ctx._ck(lib().hg_read_adjacent_moments(self.h, _p(sites), _p(mom)))
        return sites[:m], mom[:m]

    def state(self):
        """Raw F_t, shape (19, n): float32, float16, or bf16 as uint16 bit patterns."""
        dt = {0: np.float32, 1: np.float16, 2: np.uint16}[self.ctx.storage]
        out = np.zeros((19, self.n), dt)
        self.ctx._ck(lib().hg_read_state(self.h, _p(out)))
        return out

    def state_bytes(self):
        b = C.c_int64()
        self.ctx._ck(lib().hg_state_bytes(self.h, C.byref(b)))
        return b.value

    def save_state(self):
        buf = np.zeros(self.state_bytes(), np.uint8)
        self.ctx._ck(lib().hg_save_state(self.h, _p(buf), buf.size))
        return buf

    def load_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self.ctx._ck(lib().hg_load_state(self.h, _p(buf), buf.size))

    def destroy(self):
        if self.h:
            self.ctx._ck(lib().hg_domain_destroy(self.h))
            self.h = None
            self.ctx.domains.remove(self)


class Split:
    """A domain cut into partitions with a halo exchange every step (Section 2.2)."""

    def __init__(self, ctx: Context, xyz, iolets, n_parts, tau=0.8, boundary_weight=1.0, ordering="morton",
                 exchange="direct"):
        self.ctx = ctx
        xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
        lb = hg_lb_params()
        lb.tau = float(tau)
        lb.ordering = ORDER[ordering] if isinstance(ordering, str) else int(ordering)
        self.ordering = lb.ordering
        sp = hg_split_params(int(n_parts), EXCHANGE[exchange] if isinstance(exchange, str) else int(exchange),
                             float(boundary_weight))
        h = C.c_void_p()
        ctx._ck(lib().hg_split_create(ctx.h, _p(xyz), xyz.shape[0], iolet_struct_array(iolets), len(iolets),
                                      C.byref(lb), C.byref(sp), C.byref(h)))
        self.h = h
        self.n, self.n_iolets, self.n_parts = xyz.shape[0], len(iolets), int(n_parts)
        if not hasattr(ctx, "splits"):
            ctx.splits = []
        ctx.splits.append(self)

    def info(self, part):
        v = [C.c_int64() for _ in range(4)]
        self.ctx._ck(lib().hg_split_info(self.h, int(part), *[C.byref(x) for x in v]))
        return dict(first=v[0].value, owned=v[1].value, ghosts=v[2].value, halo_in=v[3].value)

    def step(self, n):
        self.ctx._ck(lib().hg_split_step(self.h, int(n)))

    def macroscopic(self):
        out = np.zeros((self.n, 4), np.float32)
        self.ctx._ck(lib().hg_split_read_macroscopic(self.h, _p(out)))
        return out

    def state(self):
        dt = {0: np.float32, 1: np.float16, 2: np.uint16}[self.ctx.storage]
        out = np.zeros((19, self.n), dt)
        self.ctx._ck(lib().hg_split_read_state(self.h, _p(out)))
        return out

    def iolet_stats(self):
        out = np.zeros((max(1, self.n_iolets), 3), np.float64)
        self.ctx._ck(lib().hg_split_read_iolet_stats(self.h, _p(out)))
        return out[: self.n_iolets]

    def boundary_values(self):
        out = np.zeros(max(1, self.n_iolets), np.float32)
        self.ctx._ck(lib().hg_split_read_boundary_values(self.h, _p(out)))
        return out[: self.n_iolets]

    def mass(self):
        out = C.c_double()
        self.ctx._ck(lib().hg_split_mass(self.h, C.byref(out)))
        return out.value

    def destroy(self):
        if self.h:
            self.ctx._ck(lib().hg_split_destroy(self.h))
            self.h = None
            self.ctx.splits.remove(self)
