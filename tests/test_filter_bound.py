"""Host check of the tensor-core NEAREST filter's error bound (no GPU).

The large-batch NEAREST kernels evaluate the expansion
    e(q, x) = |q|^2 + |x|^2 - 2 q.x
as one contraction with low-precision operands,
    A[q] = (-2 q, 1, |q|^2),  B[x] = (x, |x|^2 (1 - kTc), 1),
and skip a vertex when that value exceeds a bound built from the exact FP32
squared distance d2 of an admissible vertex:
    lim = (d2 2^2s (1 + 4 (D + 2) u) + kTq |q|^2 + kAbs) (1 + 4 u).
Results are exact only if the value computed for the true nearest vertex can
never exceed the bound built from its own distance.  This test emulates the
operand rounding of both forms in numpy and checks that inequality, with the
constants read from the kernel source:

- FP16 (up to 14 coordinates): exact power-of-two scaling that puts the
  largest magnitude in [8, 16), round to nearest, operands below 2^-14 also
  tried flushed to zero;
- TF32 (more coordinates): truncation of the low 13 mantissa bits;

products exact, the sum in float64 plus the kernels' allowance for FP32
accumulation (2^-14 of sum |a_k b_k|).  The exact FP32 distance is taken at
its smallest possible value, d2 (1 - 4 (D + 2) u).  Without its safety
terms the same check must fail (the test has teeth)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2609_30644_gb300", "csrc", "nearest.cu")
U = 2.0 ** -24


def _const(name):
    m = re.search(r"constexpr float %s = ([0-9.]+)f / ([0-9.]+)f;" % name, open(SRC).read())
    assert m, name
    return float(m.group(1)) / float(m.group(2))


K = {n: _const(n) for n in ("kTc", "kTq", "kTc16", "kTq16", "kAbs16")}


def _f32_norm2(v):
    acc = np.zeros(v.shape[0], np.float32)
    for d in range(v.shape[1]):
        acc = (acc + v[:, d] * v[:, d]).astype(np.float32)
    return acc


def _fp16(v, flush):
    h = np.asarray(v, np.float32).astype(np.float16).astype(np.float64)
    if flush:
        h[np.abs(h) < 2.0 ** -14] = 0.0
    return h


def _tf32(v):
    b = np.asarray(v, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32).astype(np.float64)


def _excess(q, x, form, flush=False, widen=True):
    """Computed filter value minus the bound built from the true distance
    (both in the kernel's units); <= 0 everywhere is the requirement.
    widen=False drops every safety term (the vertex-side fold, the query-side
    and absolute widening, the accumulation allowance)."""
    q = np.asarray(q, np.float32)
    x = np.asarray(x, np.float32)
    D = q.shape[1]
    d2 = ((q.astype(np.float64) - x.astype(np.float64)) ** 2).sum(1)
    kC1 = 4.0 * (D + 2) * U
    if form == "fp16":
        mx = float(max(np.abs(q).max(), np.abs(x).max()))
        ex = np.frexp(mx)[1]
        sc = np.float32(2.0 ** (4 - ex))
        qs, xs = (q * sc).astype(np.float32), (x * sc).astype(np.float32)
        kTc, kTq_, kAbs, rnd = K["kTc16"], K["kTq16"], K["kAbs16"], (lambda v: _fp16(v, flush))
        scale2 = float(sc) ** 2
    else:
        qs, xs = q, x
        kTc, kTq_, kAbs, rnd, scale2 = K["kTc"], K["kTq"], 0.0, _tf32, 1.0
    if not widen:
        kTc, kTq_, kAbs = 0.0, 0.0, 0.0
    qn = _f32_norm2(qs)
    xn = (_f32_norm2(xs) * np.float32(1.0 - kTc)).astype(np.float32)
    A = np.concatenate([rnd(-2.0 * qs), np.ones((len(q), 1)), rnd(qn)[:, None]], 1)
    B = np.concatenate([rnd(xs), rnd(xn)[:, None], np.ones((len(q), 1))], 1)
    prod = A * B
    S = prod.sum(1) + (2.0 ** -14 * np.abs(prod).sum(1) if widen else 0.0)
    d2_f32_low = d2 * (1.0 - kC1)
    lim = (d2_f32_low * scale2 * (1.0 + kC1) + kTq_ * qn.astype(np.float64) + kAbs) * (1.0 + 4 * U)
    return S - lim


def _cases(D, n, rng):
    box = rng.uniform(-2.9, 2.9, (2, n, D)).astype(np.float32)
    near = box[0] + rng.normal(0, 1e-3, (n, D)).astype(np.float32)   # tiny distances
    yield "box", box[0], box[1]
    yield "near", box[0], near
    yield "same", box[0], box[0].copy()                                # d = 0
    yield "offset", box[0] + 1000.0, near + 1000.0                    # large norms
    tiny = (box * 1e-6).astype(np.float32)
    tiny[:, :, 0] = box[:, :, 0]                                       # mixed magnitudes
    yield "mixed", tiny[0], tiny[1]
    yield "small", (box[0] * 1e-12).astype(np.float32), (near * 1e-12).astype(np.float32)
    big = box.copy()
    big[:, :, D // 2] *= 1e15
    yield "big", big[0], big[1]


@pytest.mark.parametrize("D", [3, 6, 7, 14])
@pytest.mark.parametrize("flush", [False, True])
def test_fp16_filter_bound(D, flush):
    rng = np.random.default_rng(D + 100 * flush)
    for name, q, x in _cases(D, 20000, rng):
        ex = _excess(q, x, "fp16", flush=flush)
        assert ex.max() <= 0.0, (name, float(ex.max()))


@pytest.mark.parametrize("D", [21, 28])
def test_tf32_filter_bound(D):
    rng = np.random.default_rng(D)
    for name, q, x in _cases(D, 20000, rng):  # all inside the [2^-60, 2^60] rule
        ex = _excess(q, x, "tf32")
        assert ex.max() <= 0.0, (name, float(ex.max()))


@pytest.mark.parametrize("form,D", [("fp16", 14), ("tf32", 28)])
def test_bound_without_widening_fails(form, D):
    """Without its safety terms the same check fails: a query placed on a
    vertex (true value 0) gets a positive computed value from operand rounding
    alone, so the inequality above is not vacuous."""
    rng = np.random.default_rng(7)
    q = rng.uniform(-2.9, 2.9, (20000, D)).astype(np.float32)
    assert _excess(q, q.copy(), form).max() <= 0.0
    assert _excess(q, q.copy(), form, widen=False).max() > 0.0


# ----------------------------------------------------------------------------
# FP32 filter on the FMA pipe (nearest_f32_kernel, the default)
# ----------------------------------------------------------------------------
# acc = xn + sum_d (-2 q_d) x_d by a chain of fused multiply-adds in FP32,
# xn = fl(|x|^2) (1 - 4 gamma), gamma = kG (D + 2) u; a pair passes when
#   acc <= T = fl_up(fl(fmaf(d2, 1 + kC1, kQ (D + 2) u qn)) (1 + 4 u) - qn).

def _f32_const(pattern):
    m = re.search(pattern, open(SRC).read())
    assert m, pattern
    return float(m.group(1))


KG = _f32_const(r"constexpr float kF32G = ([0-9.]+)f \* 5\.9604645e-8f;")
KQ = _f32_const(r"fmaf\(d2, 1\.f \+ kC1, ([0-9.]+)f \* kG \* qn\)") * KG


def _fma32(a, b, c):
    """FP32 fused multiply-add: the product of two floats is exact in float64,
    the sum is rounded once more there, then to float32 (the extra float64
    rounding is far below the allowances checked)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _excess_f32(q, x, widen=True):
    q = np.asarray(q, np.float32)
    x = np.asarray(x, np.float32)
    D = q.shape[1]
    kC1 = 4.0 * (D + 2) * U
    gamma = KG * (D + 2) * U if widen else 0.0
    kq = KQ * (D + 2) * U if widen else 0.0
    n2 = np.zeros(len(x), np.float32)
    for d in range(D):
        n2 = _fma32(x[:, d], x[:, d], n2)
    xn = (n2 * np.float32(1.0 - 4.0 * gamma)).astype(np.float32)
    acc = xn
    for d in range(D):
        acc = _fma32((np.float32(-2.0) * q[:, d]).astype(np.float32), x[:, d], acc)
    qn = np.zeros(len(q), np.float32)
    for d in range(D):
        qn = _fma32(q[:, d], q[:, d], qn)
    d2 = ((q.astype(np.float64) - x.astype(np.float64)) ** 2).sum(1)
    d2_f32_low = d2 * (1.0 - kC1)   # the exact formula's smallest possible value
    T = (d2_f32_low * (1.0 + kC1) + kq * qn.astype(np.float64)) * (1.0 + 4 * U) - qn
    return acc.astype(np.float64) - T


@pytest.mark.parametrize("D", [3, 6, 7, 14, 21, 28])
def test_fp32_filter_bound(D):
    rng = np.random.default_rng(300 + D)
    for name, q, x in _cases(D, 20000, rng):  # all inside the [2^-60, 2^60] rule
        ex = _excess_f32(q, x)
        assert ex.max() <= 0.0, (name, float(ex.max()))


def test_fp32_bound_without_widening_fails():
    """Without the fold of |x|^2 and the query-side widening, a query placed
    on a vertex far from the origin already fails the check: rounding alone."""
    rng = np.random.default_rng(8)
    q = (rng.uniform(-2.9, 2.9, (20000, 14)) + 1000.0).astype(np.float32)
    assert _excess_f32(q, q.copy()).max() <= 0.0
    assert _excess_f32(q, q.copy(), widen=False).max() > 0.0
