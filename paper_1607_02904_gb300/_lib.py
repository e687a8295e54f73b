"""ctypes binding of the C ABI in include/tersoff.h (argument marshalling only).

Every array handed to the library is a contiguous CUDA torch tensor (device
memory and streams come from PyTorch); nothing is computed here. If the shared
library cannot be built or loaded the import fails loudly: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

OK = 0
E_INVALID_ARG = 1
E_BOX_TOO_SMALL = 2
E_NEIGH_OVERFLOW = 3
E_NONFINITE = 4
E_TIMEOUT = 5
E_CUDA = 6
E_STATE = 7
FP64 = 0
MIXED = 1
SCATTER_GATHER = 0
SCATTER_ATOMIC = 1
NPARAM = 14
NOALLOC_MAX_ATOMS = 65536
REBUILD_ON_SKIN = -1
ABLATE_NO_SHORT = 1
ABLATE_GENERAL = 2
ABLATE_FP32_SUMS = 4
ABLATE_FASTFWD = 8
ABLATE_COMP_ATOM_SUMS = 16

_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIG = {
    "tersoff_create": ([ctypes.POINTER(_P), _I], _I),
    "tersoff_destroy": ([_P], _I),
    "tersoff_last_error": ([_P], ctypes.c_char_p),
    "tersoff_set_precision": ([_P, _I], _I),
    "tersoff_params": ([_P, _I, _P], _I),
    "tersoff_neighbor_build": ([_P, _P, _P, _I, _P, _D, _P], _I),
    "tersoff_neighbor_build_batched": ([_P, _P, _P, _I, _P, _P, _I, _D, _P], _I),
    "tersoff_compute_batched": ([_P, _P, _I, _P, _P, _P, _P], _I),
    "tersoff_neighbor_capacity": ([_P, _P, _P], _I),
    "tersoff_set_neighbor_capacity": ([_P, _I], _I),
    "tersoff_neighbor_export": ([_P, _P, _P, _I, _P], _I),
    "tersoff_compute": ([_P, _P, _I, _P, _P, _P, _P], _I),
    "tersoff_compute_peratom": ([_P, _P, _I, _P, _P], _I),
    "tersoff_compute_noalloc": ([_P, _P, _I, _P, _P, _P, _P], _I),
    "tersoff_backward": ([_P, _P, _I, _P, _P, _P, _P, _P], _I),
    "tersoff_md_step": ([_P, _P, _P, _P, _I, _P, _D, _I, _I, _P, _P], _I),
    "tersoff_md_step_host": ([_P, _P, _P, _P, _I, _P, _D, _I, _I, _P, _P], _I),
    "tersoff_launch_count": ([_P, _P], _I),
    "tersoff_md_rebuilds": ([_P, _P], _I),
    "tersoff_autotune": ([_P, _P, _P, _I, _P, _D, _I, _P], _I),
    "tersoff_autotune_summary": ([_P], ctypes.c_char_p),
    "tersoff_set_launch": ([_P, _I, _I, _I], _I),
    "tersoff_set_lanes": ([_P, _I], _I),
    "tersoff_set_ablation": ([_P, _I], _I),
    "tersoff_set_timing": ([_P, _I], _I),
    "tersoff_set_graphs": ([_P, _I], _I),
    "tersoff_set_scatter": ([_P, _I], _I),
    "tersoff_timing": ([_P, _I, _P, _P], _I),
    "tersoff_pipe_peaks": ([_P, _P], _I),
    "tersoff_halo_pack": ([_P, _P, _P, _P, _I, _I, _P, _I, _P, _P, _P, _P, _P, _P], _I),
    "tersoff_checkpoint_save": ([_P, ctypes.c_char_p, _P, _P, _P, _I, ctypes.c_longlong, _P], _I),
    "tersoff_checkpoint_info": ([ctypes.c_char_p, _P, _P], _I),
    "tersoff_checkpoint_load": ([_P, ctypes.c_char_p, _P, _P, _P, _P, _I, _P, _P], _I),
}


class TersoffError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tersoff status {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load():
    """Load (building first if needed) libtersoff_gb300.so and bind symbols."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIG.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def declared_symbols():
    """Entry points declared in include/tersoff.h (parsed from the header)."""
    import re
    hdr = os.path.join(os.path.dirname(_build.HERE), "include", "tersoff.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(tersoff_\w+)\(", text, re.M)))


def pipe_peaks(stream=None):
    """Measured arithmetic peaks of the current device (tersoff_pipe_peaks):
    dict of FP32 and FP64 TFLOP/s, rsqrt / ex2 / lg2 rates (1e12 ops/s) and the
    multiprocessor count."""
    lib = load()
    out = (_D * 6)()
    st = lib.tersoff_pipe_peaks(out, _stream(stream))
    if st != OK:
        raise TersoffError(st, "tersoff_pipe_peaks failed")
    keys = ("fp32_tflops", "fp64_tflops", "rsqrt_tops", "ex2_tops", "lg2_tops", "sms")
    return dict(zip(keys, [float(v) for v in out]))


def checkpoint_info(path):
    """(n, n_species) of a checkpoint file (tersoff_checkpoint_info)."""
    lib = load()
    n, ns = _I(), _I()
    st = lib.tersoff_checkpoint_info(os.fsencode(path), ctypes.byref(n), ctypes.byref(ns))
    if st != OK:
        raise TersoffError(st, f"{path!s}: not a readable checkpoint")
    return n.value, ns.value


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """One tersoff_ctx. Methods mirror the C entry points of the same names."""

    def __init__(self, precision=MIXED):
        self.lib = load()
        h = _P()
        st = self.lib.tersoff_create(ctypes.byref(h), int(precision))
        if st != OK:
            raise TersoffError(st, "tersoff_create failed")
        self.h = h
        self.n = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.tersoff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            msg = self.lib.tersoff_last_error(self.h)
            raise TersoffError(st, msg.decode() if msg else "")

    def set_precision(self, precision):
        self._check(self.lib.tersoff_set_precision(self.h, int(precision)))

    def params(self, table):
        """table: host float64 array-like of n_species^3 * 14 values."""
        import numpy as np
        t = np.ascontiguousarray(table, dtype=np.float64).ravel()
        ns = round((t.size // NPARAM) ** (1.0 / 3.0))
        assert ns ** 3 * NPARAM == t.size, "table size must be n_species^3 * 14"
        self._check(self.lib.tersoff_params(self.h, ns, t.ctypes.data_as(_P)))
        self.ns = ns

    def neighbor_build(self, x, types, box, r_list, stream=None):
        import numpy as np
        b = np.ascontiguousarray(box, dtype=np.float64)
        self.n = int(x.shape[0])
        self._check(self.lib.tersoff_neighbor_build(self.h, _ptr(x), _ptr(types), self.n,
                                                    b.ctypes.data_as(_P), float(r_list),
                                                    _stream(stream)))

    def neighbor_build_batched(self, x, types, offsets, boxes, r_list, stream=None):
        """offsets: host ints (n_systems + 1); boxes: host (n_systems, 3)."""
        import numpy as np
        off = np.ascontiguousarray(offsets, dtype=np.int32)
        bx = np.ascontiguousarray(boxes, dtype=np.float64)
        self.n = int(x.shape[0])
        self.n_sys = int(off.size - 1)
        self._check(self.lib.tersoff_neighbor_build_batched(
            self.h, _ptr(x), _ptr(types), self.n, off.ctypes.data_as(_P), bx.ctypes.data_as(_P),
            self.n_sys, float(r_list), _stream(stream)))

    def compute_batched(self, x, energies=None, forces=None, virials=None, stream=None):
        self._check(self.lib.tersoff_compute_batched(self.h, _ptr(x), int(x.shape[0]),
                                                     _ptr(energies), _ptr(forces), _ptr(virials),
                                                     _stream(stream)))

    def neighbor_capacity(self):
        cap = _I()
        mx = _I()
        self._check(self.lib.tersoff_neighbor_capacity(self.h, ctypes.byref(cap),
                                                       ctypes.byref(mx)))
        return cap.value, mx.value

    def set_neighbor_capacity(self, cap):
        self._check(self.lib.tersoff_set_neighbor_capacity(self.h, int(cap)))

    def halo_pack(self, x, types, ids, axis, geo, cap, x_local, send_x, send_t, send_id,
                  counts, stream=None):
        """tersoff_halo_pack: geo holds the 9 host doubles (L, lo, hi, r_ghost,
        frame, shift_lower, frame_lower, shift_upper, frame_upper); the output
        tensors are the caller's."""
        g = (_D * 9)(*[float(v) for v in geo])
        self._check(self.lib.tersoff_halo_pack(
            self.h, _ptr(x), _ptr(types), _ptr(ids), int(x.shape[0]), int(axis), g, int(cap),
            _ptr(x_local), _ptr(send_x), _ptr(send_t), _ptr(send_id), _ptr(counts),
            _stream(stream)))

    def neighbor_export(self, cap, stream=None):
        import torch
        cnt = torch.empty(self.n, dtype=torch.int32, device="cuda")
        nbr = torch.empty((self.n, cap), dtype=torch.int32, device="cuda")
        st = self.lib.tersoff_neighbor_export(self.h, _ptr(cnt), _ptr(nbr), int(cap),
                                              _stream(stream))
        if st not in (OK, E_NEIGH_OVERFLOW):
            self._check(st)
        return cnt, nbr, st

    def compute(self, x, energy=None, forces=None, virial=None, stream=None):
        self._check(self.lib.tersoff_compute(self.h, _ptr(x), int(x.shape[0]), _ptr(energy),
                                             _ptr(forces), _ptr(virial), _stream(stream)))

    def backward(self, x, gE, gF=None, grad_x=None, grad_table=None, stream=None):
        """gE: device float64 (1,) (one per system in batch mode); gF: device
        (N, 3) or None. Writes grad_x = d/dx [gE E + sum gF . F] = -gE F - H gF
        (H the Hessian; -gE F alone when gF is None) and grad_table =
        d/dtheta [gE E + sum gF . F] (flat table layout); either may be None."""
        self._check(self.lib.tersoff_backward(self.h, _ptr(x), int(x.shape[0]), _ptr(gE), _ptr(gF),
                                              _ptr(grad_x), _ptr(grad_table), _stream(stream)))

    def compute_noalloc(self, x, energy=None, forces=None, virial=None, stream=None):
        """tersoff_compute without any memory allocation in the call (fixed
        scratch inside the library; at most NOALLOC_MAX_ATOMS atoms; calls
        that overlap on the GPU share that scratch and race)."""
        self._check(self.lib.tersoff_compute_noalloc(self.h, _ptr(x), int(x.shape[0]),
                                                     _ptr(energy), _ptr(forces), _ptr(virial),
                                                     _stream(stream)))

    def compute_peratom(self, x, eatom, stream=None):
        self._check(self.lib.tersoff_compute_peratom(self.h, _ptr(x), int(x.shape[0]),
                                                     _ptr(eatom), _stream(stream)))

    def md_step(self, x, v, f, mass, dt, nsteps, rebuild_every, thermo=None, stream=None):
        import numpy as np
        m = np.ascontiguousarray(mass, dtype=np.float64)
        self._check(self.lib.tersoff_md_step(self.h, _ptr(x), _ptr(v), _ptr(f), int(x.shape[0]),
                                             m.ctypes.data_as(_P), float(dt), int(nsteps),
                                             int(rebuild_every), _ptr(thermo), _stream(stream)))

    def checkpoint_save(self, path, x, v, f, step=0, stream=None):
        """Writes the MD state (x, v, f device tensors, the context's species,
        table, box, list radius, precision and rebuild phase) to `path`."""
        self._check(self.lib.tersoff_checkpoint_save(self.h, os.fsencode(path), _ptr(x), _ptr(v),
                                                     _ptr(f), int(x.shape[0]), int(step),
                                                     _stream(stream)))

    def checkpoint_load(self, path, x, v, f, types, stream=None):
        """Restores a checkpoint into this context and the device tensors x, v,
        f (N x 3 float64) and types (N int32); returns the saved step."""
        step = ctypes.c_longlong()
        self._check(self.lib.tersoff_checkpoint_load(self.h, os.fsencode(path), _ptr(x), _ptr(v),
                                                     _ptr(f), _ptr(types), int(x.shape[0]),
                                                     ctypes.byref(step), _stream(stream)))
        return step.value

    def md_step_host(self, x, v, f, mass, dt, nsteps, rebuild_every, thermo=None, stream=None):
        """x, v, f, thermo: host (ideally pinned) float64 torch tensors."""
        import numpy as np
        m = np.ascontiguousarray(mass, dtype=np.float64)
        self._check(self.lib.tersoff_md_step_host(self.h, _ptr(x), _ptr(v), _ptr(f),
                                                  int(x.shape[0]), m.ctypes.data_as(_P),
                                                  float(dt), int(nsteps), int(rebuild_every),
                                                  _ptr(thermo), _stream(stream)))

    def set_scatter(self, mode):
        self._check(self.lib.tersoff_set_scatter(self.h, int(mode)))

    def set_graphs(self, enable=True):
        self._check(self.lib.tersoff_set_graphs(self.h, int(bool(enable))))

    def set_timing(self, enable=True):
        self._check(self.lib.tersoff_set_timing(self.h, int(bool(enable))))

    def timing(self, kind):
        """(total_ms, launches) of kind 0 force kernel, 1 neighbour build, 2 integrate."""
        ms = _D()
        cnt = ctypes.c_longlong()
        self._check(self.lib.tersoff_timing(self.h, int(kind), ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, cnt.value

    def autotune(self, x, v=None, mass=None, dt=0.001, steps=10, stream=None):
        """Time the launch options on this system (MD steps on copies when v is
        given, else force evaluations) and keep the fastest; returns the summary."""
        import numpy as np
        m = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
        self._check(self.lib.tersoff_autotune(self.h, _ptr(x), _ptr(v), int(x.shape[0]),
                                              None if m is None else m.ctypes.data_as(_P),
                                              float(dt), int(steps), _stream(stream)))
        return self.autotune_summary()

    def set_launch(self, waves=0, split=-1, block=256):
        self._check(self.lib.tersoff_set_launch(self.h, int(waves), int(split), int(block)))

    def set_lanes(self, lanes=0):
        """Lanes per atom of the main force launch: 0 automatic, 1 or 4."""
        self._check(self.lib.tersoff_set_lanes(self.h, int(lanes)))

    def set_ablation(self, flags):
        """ABLATE_NO_SHORT | ABLATE_GENERAL | ABLATE_FP32_SUMS | ABLATE_FASTFWD |
        ABLATE_COMP_ATOM_SUMS, for measuring the design choices."""
        self._check(self.lib.tersoff_set_ablation(self.h, int(flags)))

    def autotune_summary(self):
        return self.lib.tersoff_autotune_summary(self.h).decode()

    def md_rebuilds(self):
        """Neighbour rebuilds during the last md_step call."""
        c = _I()
        self._check(self.lib.tersoff_md_rebuilds(self.h, ctypes.byref(c)))
        return c.value

    def launch_count(self):
        c = ctypes.c_longlong()
        self._check(self.lib.tersoff_launch_count(self.h, ctypes.byref(c)))
        return c.value
