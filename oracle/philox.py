"""Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).

TEST INFRASTRUCTURE: part of the FP64 CPU oracle.

The random numbers Prony's method draws -- the combination weights mu of
C_mu (Algorithm 1, the step after the S_l) and the starting blocks U_0, V_0
of the block power method (Algorithm 3) -- are defined as functions of a
64-bit seed through this published generator, so that the oracle and the
GPU library (which carries its own implementation) draw the same numbers
without sharing code.

Convention (both sides):
  key      = (seed, stream)         stream: STREAM_MU, STREAM_V0, STREAM_U0
  counter  = (index, 0, 0, 0)       one 4x64-bit block per drawn complex number
  uniform  u_w = ((w >> 11) + 0.5) * 2^-53   in (0, 1)
  complex standard normal (E|z|^2 = 1) by Box-Muller from words 0 and 1:
           z = sqrt(-log u_0) * exp(2 pi i u_1)
"""
from __future__ import annotations

import numpy as np

_M0 = 0xD2E7470EE14C6C93
_M1 = 0xCA5A826395121157
_W0 = 0x9E3779B97F4A7C15
_W1 = 0xBB67AE8584CAA73B
_MASK = (1 << 64) - 1

STREAM_MU = 0x4D55      # "MU"
STREAM_V0 = 0x5630      # "V0"
STREAM_U0 = 0x5530      # "U0"


def philox4x64_10(counter, key):
    """One Philox4x64 block with 10 rounds, on Python integers."""
    c0, c1, c2, c3 = (int(v) & _MASK for v in counter)
    k0, k1 = (int(v) & _MASK for v in key)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> 64, p0 & _MASK
        hi1, lo1 = p1 >> 64, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def _uniform(w: int) -> float:
    return ((w >> 11) + 0.5) * (2.0 ** -53)


def complex_normal(seed: int, stream: int, index: int) -> complex:
    w = philox4x64_10((index, 0, 0, 0), (seed, stream))
    u0, u1 = _uniform(w[0]), _uniform(w[1])
    return complex(np.sqrt(-np.log(u0)) * np.exp(2j * np.pi * u1))


def complex_normal_block_scalar(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols matrix, entry (i, j) drawn with counter index i*cols + j (Python integers)."""
    out = np.empty((rows, cols), dtype=np.complex128)
    for i in range(rows):
        for j in range(cols):
            out[i, j] = complex_normal(seed, stream, i * cols + j)
    return out


def _mulhilo64(a: np.ndarray, b: int):
    """Full 64x64 -> 128-bit product of uint64 arrays by a constant, from 32-bit halves."""
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    a0, a1 = a & m32, a >> s32
    b0, b1 = np.uint64(b & 0xFFFFFFFF), np.uint64(b >> 32)
    p00, p01, p10, p11 = a0 * b0, a0 * b1, a1 * b0, a1 * b1
    mid = (p00 >> s32) + (p01 & m32) + (p10 & m32)
    hi = p11 + (p01 >> s32) + (p10 >> s32) + (mid >> s32)
    lo = (mid << s32) | (p00 & m32)
    return hi, lo


def philox4x64_10_vec(counter0: np.ndarray, key) -> tuple:
    """Philox4x64-10 of counters (counter0, 0, 0, 0) for an array of counter0, numpy uint64."""
    with np.errstate(over="ignore"):
        c0 = counter0.astype(np.uint64)
        c1 = np.zeros_like(c0)
        c2 = np.zeros_like(c0)
        c3 = np.zeros_like(c0)
        k0, k1 = int(key[0]) & _MASK, int(key[1]) & _MASK
        for _ in range(10):
            hi0, lo0 = _mulhilo64(c0, _M0)
            hi1, lo1 = _mulhilo64(c2, _M1)
            c0, c1, c2, c3 = hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def complex_normal_block(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols matrix, entry (i, j) drawn with counter index i*cols + j."""
    idx = np.arange(rows * cols, dtype=np.uint64)
    w0, w1, _, _ = philox4x64_10_vec(idx, (seed, stream))
    u0 = ((w0 >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    u1 = ((w1 >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    z = np.sqrt(-np.log(u0)) * np.exp(2j * np.pi * u1)
    return z.reshape(rows, cols)


def draw_mu(seed: int, d: int) -> np.ndarray:
    """mu in C^d with ||mu||_2 = 1 (Algorithm 1: random point of the unit sphere S_C^{d-1})."""
    mu = np.array([complex_normal(seed, STREAM_MU, l) for l in range(d)])
    return mu / np.linalg.norm(mu)
