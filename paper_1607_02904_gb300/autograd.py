"""Energy and forces as differentiable functions of positions and parameters.

``energy_forces(system, x, table)`` returns (E, F) from the CUDA library's
``tersoff_compute``; its backward runs the library's adjoint kernel
(``tersoff_backward``): the gradient of ``gE E + sum_a gF_a . F_a`` with respect
to the parameter table and with respect to the positions (``-gE F`` plus the
Hessian-vector product ``-H gF``), so a loss on energies and forces can be
differentiated in both. The returned gradients are not themselves
differentiable (no double backward). Everything here marshals arguments; the
arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch
from torch.autograd.function import once_differentiable

from ._lib import MIXED, NPARAM, Context


class TersoffSystem:
    """One periodic system: a library context holding the species, box,
    neighbour list and the parameter table last uploaded.

    types: (N,) int species; box: 3 edges (A); r_list: cutoff plus skin (A).
    The list is rebuilt whenever a new table is uploaded (the filter radii
    depend on the cutoffs) or ``rebuild(x)`` is called. A table is uploaded
    when it is a different tensor, or the same tensor modified in place, than
    at the last call (its values are then compared on the host); an unchanged
    table costs no device work, so forward and backward can be captured in a
    CUDA graph."""

    energies_shape = ()

    def __init__(self, types, box, r_list, precision=MIXED, device=None):
        self.device = torch.device(device if device is not None else "cuda")
        self.ctx = Context(precision)
        self.types = torch.as_tensor(np.asarray(types), dtype=torch.int32,
                                     device=self.device).contiguous()
        self.box = np.ascontiguousarray(box, dtype=np.float64)
        self.r_list = float(r_list)
        self._table = None
        self._key = None
        self.version = 0
        self.ntable = 0

    def load(self, x, table):
        """Upload ``table`` (if it changed) and build the list at x."""
        key = (table.data_ptr(), str(table.device), table._version, tuple(table.shape))
        if key == self._key:
            return
        t = table.detach().to("cpu", torch.float64).contiguous().numpy().ravel()
        if self._table is None or t.shape != self._table.shape or not np.array_equal(t, self._table):
            self.ctx.params(t)
            self._table = t.copy()
            self.ntable = t.size
            self.version += 1
            self.rebuild(x)
        self._key = key

    def rebuild(self, x):
        self.ctx.neighbor_build(x.detach().contiguous(), self.types, self.box, self.r_list)

    def evaluate(self, x, e, f):
        self.ctx.compute(x, e, f)


class TersoffBatch(TersoffSystem):
    """Independent periodic systems in one context: the atoms of system s are
    rows offsets[s]:offsets[s+1] of x; boxes (n_systems, 3). Energies are per
    system."""

    def __init__(self, types, offsets, boxes, r_list, precision=MIXED, device=None):
        super().__init__(types, np.zeros(3), r_list, precision, device)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int32)
        self.boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
        self.n_systems = self.offsets.size - 1
        self.energies_shape = (self.n_systems,)

    def rebuild(self, x):
        self.ctx.neighbor_build_batched(x.detach().contiguous(), self.types, self.offsets,
                                        self.boxes, self.r_list)

    def evaluate(self, x, e, f):
        self.ctx.compute_batched(x, e, f)


class TersoffFunction(torch.autograd.Function):
    """(E, F) = f(x, table) for one ``TersoffSystem``."""

    @staticmethod
    def forward(fctx, x, table, system):
        xd = x.detach().contiguous()
        system.load(xd, table)
        ne = int(np.prod(system.energies_shape)) if system.energies_shape else 1
        e = torch.empty(ne, dtype=torch.float64, device=xd.device)
        f = torch.empty_like(xd)
        system.evaluate(xd, e, f)
        fctx.system = system
        fctx.version = system.version
        fctx.table_shape = table.shape
        fctx.table_device = table.device
        fctx.set_materialize_grads(False)
        fctx.save_for_backward(xd)
        return e.reshape(system.energies_shape), f

    @staticmethod
    @once_differentiable
    def backward(fctx, gE, gF):
        (x,) = fctx.saved_tensors
        system = fctx.system
        if system.version != fctx.version:
            raise RuntimeError("the system's parameter table changed after this forward call")
        need_x, need_t = fctx.needs_input_grad[0], fctx.needs_input_grad[1]
        dev = x.device
        ne = int(np.prod(system.energies_shape)) if system.energies_shape else 1
        if gE is None:
            ge = torch.zeros(ne, dtype=torch.float64, device=dev)
        else:
            ge = gE.reshape(ne).to(dev, torch.float64).contiguous()
        gf = None if gF is None else gF.to(dev, torch.float64).contiguous()
        gx = torch.empty_like(x) if need_x else None
        gt = torch.empty(system.ntable, dtype=torch.float64, device=dev) if need_t else None
        if need_x or need_t:
            system.ctx.backward(x, ge, gf, gx, gt)
        if gt is not None:
            gt = gt.reshape(fctx.table_shape).to(fctx.table_device)
        return gx, gt, None


def energy_forces(system: TersoffSystem, x: torch.Tensor, table: torch.Tensor):
    """Energy (0-dim; per system for a TersoffBatch) and forces (N, 3),
    differentiable in ``table`` and in ``x``."""
    return TersoffFunction.apply(x, table, system)


__all__ = ["TersoffSystem", "TersoffBatch", "TersoffFunction", "energy_forces", "NPARAM"]
