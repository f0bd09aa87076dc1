"""Numerical methods of the CUDA kernels checked against their stated error bounds, emulated on the
CPU with IEEE single precision (numpy float32; a fused multiply-add is the exact product and sum
rounded once, which float64 represents exactly for float32 operands)."""
import numpy as np

from oracle import prism_oracle as O


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def fma32(a, b, c):
    # a*b of two float32 values is exact in float64 (48 significant bits); the sum is rounded to
    # float64 once (below float32 resolution) and then to float32
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def test_transmission_phase_reduction_in_float_float():
    # the transmission kernel splits sigma (cycles per V.A) into float hi + lo, forms p = V hi, its
    # exact error e = fma(V, hi, -p) and c = (p - rint(p)) + fma(V, lo, e); c must equal the fractional
    # part of sigma V (FP64 reference) to about 2^-24 cycles
    sigma = O.interaction_constant(300.0) / (2.0 * np.pi)
    hi = f32(sigma)
    lo = f32(sigma - np.float64(hi))
    rng = np.random.Generator(np.random.PCG64(5))
    v = f32(np.concatenate([rng.random(20000) * 500.0, rng.random(20000) * 2.0e5, [0.0, 1.0, 12345.678]]))
    p = f32(np.float64(v) * np.float64(hi))
    e = fma32(v, hi, -np.float64(p))
    frac = f32(np.float64(p) - np.rint(np.float64(p)))   # exact for |p| < 2^23
    c = f32(np.float64(frac) + np.float64(fma32(v, lo, e)))
    ref = sigma * np.float64(v)
    ref -= np.rint(ref)
    err = np.abs(np.float64(c) - ref)
    err = np.minimum(err, 1.0 - err)  # a phase of +1/2 and -1/2 cycles is the same point
    assert err.max() < 2.0 ** -23
