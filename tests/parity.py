"""Error measures shared by the GPU parity tests.

The paper compares an optimised kernel with the naive one through the Frobenius norm of
the difference (Sec. 4.9) without giving a value; the tests state theirs.  Two views of
the same difference are checked:

* per quantity: for every quantity p, ||X_gpu[:, :, p] - X_ref[:, :, p]||_F divided by
  ||X_ref[:, :, p]||_F, over all elements and basis functions (a quantity with a small
  norm keeps its own scale);
* per element: for every element e, ||X_gpu[e] - X_ref[e]||_F / ||X_ref[e]||_F, and the
  maximum over e.  An error confined to one element is diluted by about sqrt(E) in the
  first view; the second one sees it at full size.

Arrays are (elements, basis functions, quantities) or lists of (basis, quantities)
arrays of different sizes (p-adaptive meshes).  `check` prints one `PARITY` line per call
(name, both maxima, both bounds) so that a run with `-s` records the measured errors.
"""
import numpy as np


def _stack(x):
    if isinstance(x, (list, tuple)):
        return x
    return np.asarray(x)


def per_quantity(got, ref):
    if isinstance(ref, (list, tuple)):
        g = np.concatenate([np.asarray(a) for a in got], axis=0)
        r = np.concatenate([np.asarray(a) for a in ref], axis=0)
        num = np.sqrt(((g - r) ** 2).sum(axis=0))
        den = np.sqrt((r ** 2).sum(axis=0))
    else:
        num = np.sqrt(((got - ref) ** 2).sum(axis=(0, 1)))
        den = np.sqrt((ref ** 2).sum(axis=(0, 1)))
    return num / np.where(den > 0, den, 1.0)


def per_element(got, ref):
    if isinstance(ref, (list, tuple)):
        num = np.array([np.linalg.norm(np.asarray(a) - np.asarray(b)) for a, b in zip(got, ref)])
        den = np.array([np.linalg.norm(b) for b in ref])
    else:
        num = np.sqrt(((got - ref) ** 2).sum(axis=(1, 2)))
        den = np.sqrt((ref ** 2).sum(axis=(1, 2)))
    return num / np.where(den > 0, den, 1.0)


def increment(x, base):
    if isinstance(x, (list, tuple)):
        return [np.asarray(a) - np.asarray(b) for a, b in zip(x, base)]
    return x - base


def check(name, got, ref, tol_quantity, tol_element, base=None):
    """Asserts both views of got - ref within their bounds; with `base`, the increments
    got - base and ref - base are compared instead (the part of Q a step changes)."""
    got, ref = _stack(got), _stack(ref)
    if base is not None:
        got, ref = increment(got, base), increment(ref, base)
    eq = float(per_quantity(got, ref).max())
    ee = float(per_element(got, ref).max())
    print(f"PARITY {name}: per-quantity {eq:.3e} (bound {tol_quantity:.1e}), "
          f"per-element {ee:.3e} (bound {tol_element:.1e})")
    assert eq < tol_quantity, (name, "per quantity", eq, tol_quantity)
    assert ee < tol_element, (name, "per element", ee, tol_element)
    return eq, ee


# ------------------------------------------------------------------------- bounds
# FP64: 1e-12 on Q and on I, 1e-11 on the increment Q_new - Q (the increment is about a
# tenth of Q, so its relative error is about ten times that of Q); measured at most
# 1.2e-14 (per element) over orders 2..7 and 1M tets.
F64 = 1e-12
F64_INC = 1e-11
# FP32 contractions (unit roundoff u = 2^-24 = 6.0e-8).  The increment passes through the
# CK chain (N derivatives: sparse rows of up to ~60 products, a 3 x 9 mixing), the volume,
# the face projections and the lifting, each rounding at about u sqrt(n) relative; the
# measured maxima over orders 2..7 (tests below and 400 sampled elements of 1M tets) are
# 3.4e-7 = 5.7 u per quantity and 4.7e-7 = 7.8 u per element.  The time integral is
# accumulated in binary64 and dominated by its exact c0 Q term: 1.2e-8 / 1.3e-8.
# Bounds: about nine times the measured maxima (50 u and 67 u on the increment).
F32_INC, F32_INC_EL = 3e-6, 4e-6
F32_I, F32_I_EL = 1e-7, 1.2e-7
# Split-bf16 tensor cores: every product with a global matrix carries about 2^-16 = 1.5e-5
# relative error (the dropped lo x lo term; hi + lo holds 16 significant bits), errors of
# a sum average out: measured 1.1e-5 per quantity and 1.7e-5 per element on the
# increment, 4.4e-6 / 7.0e-6 on the time integral (N(0,1) DOFs, orders 2..6).  Bounds:
# about nine times these (6.5 and 10 times 2^-16 on the increment).
TC_INC, TC_INC_EL = 1e-4, 1.5e-4
TC_I, TC_I_EL = 4e-5, 6e-5
# 27 quantities, FP32 contractions: measured 2.8e-7 per quantity and 5.1e-8 per element
# on the increment (orders 2..7, random mesh and 3 steps on the jittered mesh), 2.1e-8 /
# 3.2e-8 on the time integral; the per-element figure is lower than in the elastic case
# because the anelastic functions, which carry most of an element's norm, see only a few
# roundings per step.  Bounds about nine times these.
VE_F32_INC, VE_F32_INC_EL = 2.5e-6, 5e-7
VE_F32_I, VE_F32_I_EL = 2e-7, 3e-7
# 27 quantities, split-bf16 tensor cores for the elastic rows (the anelastic functions in
# FP32 from the same accumulators): measured 8.6e-6 per quantity and 3.5e-7 per element on
# the increment (orders 2..7, random mesh and 3 steps on the jittered mesh), 3.6e-7 / 3.1e-8
# on the time integral; as in FP32 the anelastic functions carry most of an element's norm
# and see only FP32 roundings.  Bounds about nine times these.
VE_TC_INC, VE_TC_INC_EL = 8e-5, 3.5e-6
VE_TC_I, VE_TC_I_EL = 3.5e-6, 3e-7
