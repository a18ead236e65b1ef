"""Seeded synthetic persistence diagrams shaped like the paper's workloads.

Input generation only: nothing here computes any part of the W1 method.  The
oracle and the CUDA library both draw their inputs from these functions.

* uniform_exp(n, seed): birth b ~ U[0,1], death d = min(b + p, 1) with
  p ~ Exp(mean 0.05), both rounded to a 1/256 grid, float32.  About 3.5% of
  the points land on the diagonal (b == d) and are dropped by the method.
* lowerstar_u8(n, seed): 0-dimensional lower-star persistence of 512x512
  white-noise images smoothed by a Gaussian (sigma 2 px) and min-max scaled to
  uint8, pooled over successive seeded images until n points; uint8 (b, d)
  pairs with many duplicates (the 8-bit image datasets of the paper's
  experiments stand behind this shape; the datasets themselves are not used).
* mixture_f32(n, seed): b ~ U[0,1], persistence p ~ 0.95 Exp(mean 0.01) +
  0.05 U[0, 0.5], d = b + p, float32, few duplicates.
* gaussian_pd(n, seed): points of a 2D Gaussian mirrored above the diagonal
  (the synthetic Gaussian diagrams of the empirical-complexity experiment).
* db_sizes(count, seed, lo, hi): log-uniform diagram sizes in [lo, hi].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "synth_lowerstar.c")
_LIB = os.path.join(_HERE, "_lib", "libsynth.so")
_lib = None


def build_helper(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _helper():
    global _lib
    if _lib is None:
        L = C.CDLL(build_helper())
        L.synth_lowerstar_h0.restype = C.c_int64
        L.synth_lowerstar_h0.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64]
        _lib = L
    return _lib


def uniform_exp(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    b = rng.random(n)
    p = rng.exponential(0.05, n)
    d = np.minimum(b + p, 1.0)
    bd = np.stack([np.round(b * 256.0) / 256.0, np.round(d * 256.0) / 256.0], axis=1)
    return bd.astype(np.float32)


def mixture_f32(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    b = rng.random(n)
    pick = rng.random(n) < 0.95
    p = np.where(pick, rng.exponential(0.01, n), rng.random(n) * 0.5)
    return np.stack([b, b + p], axis=1).astype(np.float32)


def gaussian_pd(n: int, seed: int) -> np.ndarray:
    """Synthetic Gaussian diagram (the empirical-complexity experiment of the
    appendix): n points of a 2D Gaussian (mean (0.4, 0.6), standard deviation
    0.15 per axis, independent), each point mirrored above the diagonal
    (birth <= death), float32.  Not a persistence diagram of any filtration."""
    rng = np.random.default_rng(seed)
    x = rng.normal(0.4, 0.15, n)
    y = rng.normal(0.6, 0.15, n)
    return np.stack([np.minimum(x, y), np.maximum(x, y)], axis=1).astype(np.float32)


def _gauss_smooth(img: np.ndarray, sigma: float) -> np.ndarray:
    r = int(4 * sigma)
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    k /= k.sum()
    out = img
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r, r)
        p = np.pad(out, pad, mode="reflect")
        acc = np.zeros_like(out)
        for t in range(2 * r + 1):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(t, t + out.shape[axis])
            acc += k[t] * p[tuple(sl)]
        out = acc
    return out


def lowerstar_image(seed: int, index: int, size: int = 512) -> np.ndarray:
    rng = np.random.default_rng([seed, index])
    g = _gauss_smooth(rng.standard_normal((size, size)), 2.0)
    lo, hi = g.min(), g.max()
    u = np.floor((g - lo) / (hi - lo) * 255.0 + 0.5)
    return np.clip(u, 0, 255).astype(np.uint8)


def lowerstar_u8(n: int, seed: int, size: int = 512) -> np.ndarray:
    L = _helper()
    parts = []
    total = 0
    idx = 0
    while total < n:
        img = np.ascontiguousarray(lowerstar_image(seed, idx, size))
        buf = np.zeros((size * size, 2), np.uint8)
        m = L.synth_lowerstar_h0(img.ctypes.data, size, size, buf.ctypes.data, size * size)
        parts.append(buf[:m])
        total += m
        idx += 1
    return np.ascontiguousarray(np.concatenate(parts, axis=0)[:n])


def db_sizes(count: int, seed: int, lo: int = 100, hi: int = 50000) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), count))).astype(np.int64)


def pair_seeds(i: int):
    """Seeds of the i-th benchmark pair."""
    return 1000 + 2 * i, 1000 + 2 * i + 1
