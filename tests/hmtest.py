"""Helpers shared by the GPU parity tests: device I/O, error metrics, bounds."""

import numpy as np

from oracle import bounds as OB

UNIT = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -9, "bf16x2": 2.0 ** -17}


def torch_dev():
    import torch
    return torch.device("cuda:0")


def to_dev(X, dtype="f64"):
    """(n, r) float64 numpy -> column-major torch tensor on cuda:0 of `dtype`."""
    import torch
    td = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(X, dtype=np.float64).T)).to(torch_dev())
    return t.to(td).t()


def exact_input(X, dtype):
    """The float64 value of X after rounding to `dtype` (what the GPU actually reads)."""
    import torch
    if dtype == "f64":
        return np.asarray(X, dtype=np.float64)
    td = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    return torch.from_numpy(np.asarray(X, dtype=np.float64)).to(td).to(torch.float64).numpy()


def to_host(Y):
    import torch
    torch.cuda.synchronize()
    return Y.to(torch.float64).cpu().numpy()


def col_rel_err(Y, ref):
    """max over columns of ||Y_j - ref_j||_2 / ||ref_j||_2."""
    Y = np.asarray(Y, dtype=np.float64).reshape(ref.shape)
    num = np.linalg.norm(Y - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    den = np.where(den == 0, 1.0, den)
    return float(np.max(num / den)) if ref.size else 0.0


# Normwise gate per column for the BF16 storages: ||y - y_oracle||_2 / ||y_oracle||_2
# <= 8 u_s.  The componentwise bound alone is c_round u_s times an envelope
# that can be several times |y|, loose enough to pass a dropped level.
NORMWISE = {"bf16": 8 * 2.0 ** -9, "bf16x2": 8 * 2.0 ** -17}


class Bound(float):
    """A componentwise bound factor that remembers the storage type it was
    derived for, so that check_bound also applies that storage's normwise gate
    (sums with plain numbers keep the storage)."""

    def __new__(cls, value, storage):
        obj = float.__new__(cls, value)
        obj.storage = storage
        return obj

    def __add__(self, other):
        return Bound(float(self) + float(other), self.storage)

    __radd__ = __add__


def bound_factor(storage, kind, p, acc_len, tensor_core=False):
    """(c_round * u_s + gamma_L(u_acc)): rounded factors on the longest product chain
    (HODLR: U, V, X and the staged T; HSS: U, V, X, y-hat and the 2(p-1) translations
    and the coupling) plus the accumulations."""
    u_s = UNIT[storage]
    # Tensor-core accumulation is not assumed to round to nearest: one ulp of FP32.
    u_acc = 2.0 ** -53 if storage == "f64" else (2.0 ** -23 if tensor_core or storage in ("bf16", "bf16x2")
                                                else 2.0 ** -24)
    c_round = 5 if kind == "hodlr" else 2 * p + 6
    if storage != "f64":
        c_round += 2   # intermediates (T / x-hat / y-hat) held in float32
    if storage in ("bf16", "bf16x2"):
        c_round += 2   # the tensor-core path rounds X and Z to the storage format
    return Bound(c_round * u_s + OB.gamma(acc_len, u_acc), storage)


def acc_length(info, kind):
    m_pad, Ke, p = info["leaf_pad"], info["rank_total"], info["depth"]
    return 2 * m_pad + 2 * Ke + (p + 2) * 2 * max(Ke, 8) + 64


def check_bound(Y, ref, env, factor, what=""):
    err = np.abs(np.asarray(Y, dtype=np.float64).reshape(ref.shape) - ref)
    tol = float(factor) * env + 1e-300
    bad = err > tol
    ratio = float(np.max(err / tol)) if ref.size else 0.0
    assert not bad.any(), "%s: %d entries beyond the bound; max err/bound = %.3g" % (what, int(bad.sum()), ratio)
    gate = NORMWISE.get(getattr(factor, "storage", None))
    if gate is not None and ref.size:
        nw = col_rel_err(Y, ref)
        assert nw <= gate, "%s: normwise per-column error %.3g above %.3g" % (what, nw, gate)
    return ratio
