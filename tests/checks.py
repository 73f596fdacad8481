"""Tolerance and comparison helpers for the parity tests.

Bars (stated for these kernels):
  FP32 vector update .......... within 1 ulp of the oracle rounded to FP32
                                (bit-exact at alpha = 0.5, where y + 0.5 z is
                                a single rounding on both sides)
  FP32 dot / GEMV / SpMV ...... norm-wise relative error <= 1e-5
  FP64 (all) .................. <= 1e-12
  BF16 / FP16 storage ......... element-wise: one ulp of the storage type at
                                the oracle's value (output rounding) plus the
                                worst-case FP32 summation error n * 2^-24 *
                                sum_j |a_ij x_j| for a row of n terms; and
                                norm-wise within one unit roundoff of the
                                storage type.  Dot (FP32 output): norm-wise
                                <= 1e-5 as for FP32
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

TOL = {"f32": 1e-5, "f64": 1e-12, "bf16": 1e-5, "f16": 1e-5}
FRAC_BITS = {"f32": 23, "f64": 52, "bf16": 7, "f16": 10}
MIN_EXP = {"f32": -126, "f64": -1022, "bf16": -126, "f16": -14}


def host(t: torch.Tensor):
    """Device tensor -> stored values widened to float64 (via the oracle's widen)."""
    return oracle.widen(t.detach().cpu())


def spacing(v: np.ndarray, storage: str) -> np.ndarray:
    """Distance from |v| to the next larger value of the storage type
    (v given as float64 holding storage-type values)."""
    a = np.abs(v)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, MIN_EXP[storage])
    return np.exp2(e - FRAC_BITS[storage])


def assert_ulp(got: np.ndarray, ref_rounded: np.ndarray, storage: str, k: float = 1.0, what=""):
    diff = np.abs(got - ref_rounded)
    bound = k * spacing(ref_rounded, storage)
    bad = np.nonzero(diff > bound)[0]
    assert bad.size == 0, (f"{what}: {bad.size} elements beyond {k} ulp; first at {bad[:5]}: "
                           f"got {got[bad[:5]]}, ref {ref_rounded[bad[:5]]}")


def normwise(got: np.ndarray, ref: np.ndarray) -> float:
    nref = np.linalg.norm(ref)
    nd = np.linalg.norm(got - ref)
    return float(nd / nref) if nref > 0 else float(nd)


def assert_normwise(got, ref, storage: str, what=""):
    err = normwise(got, ref)
    assert err <= TOL[storage], f"{what}: norm-wise relative error {err:.3e} > {TOL[storage]:g}"


def assert_dot(got: float, ref: float, x: np.ndarray, y: np.ndarray, storage: str, what=""):
    scale = float(np.linalg.norm(x) * np.linalg.norm(y))
    err = abs(got - ref)
    assert err <= TOL[storage] * max(scale, 1e-300), (
        f"{what}: |dot - oracle| = {err:.3e} > {TOL[storage]:g} * ||x|| ||y|| = "
        f"{TOL[storage] * scale:.3e}")


def canary_buffer(n: int, dtype: torch.dtype, device, pad: int = 64):
    """(buffer, view): an output view of n elements with `pad` NaN-filled
    guard elements on both sides, to catch writes outside the output."""
    buf = torch.full((n + 2 * pad,), float("nan"), dtype=dtype, device=device)
    return buf, buf[pad:pad + n]


def assert_canary(buf: torch.Tensor, n: int, pad: int = 64):
    b = buf.detach().cpu()
    assert torch.isnan(b[:pad].float()).all() and torch.isnan(b[pad + n:].float()).all(), \
        "a kernel wrote outside its output"


UNIT_ROUNDOFF = {"f32": 2.0 ** -24, "f64": 2.0 ** -53, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}


def assert_reduced_sum(got: np.ndarray, ref: np.ndarray, abs_terms: np.ndarray,
                       nterms: np.ndarray, storage: str, what=""):
    """Outputs of an FP32-accumulated sum stored in BF16/FP16 (see module doc)."""
    ref_r = oracle.round_to(ref, storage)
    bound = spacing(ref_r, storage) + nterms * 2.0 ** -24 * abs_terms
    bad = np.nonzero(np.abs(got - ref_r) > bound)[0]
    assert bad.size == 0, (f"{what}: {bad.size} elements beyond the bound; first at {bad[:5]}: "
                           f"got {got[bad[:5]]}, ref {ref_r[bad[:5]]}")
    nref = np.linalg.norm(ref)
    if nref > 0:
        err = np.linalg.norm(got - ref) / nref
        assert err <= 2 * UNIT_ROUNDOFF[storage], f"{what}: norm-wise {err:.3e}"


def assert_normwise_scaled(got, ref, abs_ref, storage: str, what=""):
    """||got - ref|| <= tol * || |A| |x| ||: the scale of FP32 accumulation error
    (for outputs of very few rows, where ||y|| itself may be small because of
    cancellation inside a row)."""
    scale = float(np.linalg.norm(abs_ref))
    err = float(np.linalg.norm(got - ref))
    assert err <= TOL[storage] * max(scale, 1e-300), (
        f"{what}: ||err|| = {err:.3e} > {TOL[storage]:g} * || |A||x| || = {TOL[storage] * scale:.3e}")
