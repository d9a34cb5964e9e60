"""Exact models of the tensor-core Gram and recovery arithmetic, for tests.

The kernels document their arithmetic (kernels_gram_tc.cu): each column of Y
becomes trunc(y 2^(55 - E)), E = emax - 1022 for the column's largest biased
exponent emax, written in seven balanced base-256 digits; digit products of
levels i + j <= 7 are summed exactly and the sums are rounded to FP64 in a
fixed way. These models redo that in numpy with exact integer arithmetic
(digit products are small integers, so float64 matrix products of them are
exact too) and let the GPU tests compare bit for bit. They are written from
that description, not from the CUDA code, and share nothing with the product.
"""
import math

import numpy as np

LEVELS = 7  # the largest level i + j kept


def bexp(v):
    """Biased exponents of float64 values."""
    return (np.asarray(v, dtype=np.float64).view(np.uint64) >> np.uint64(52)).astype(np.int64) & 0x7FF


def digits55(y, emax):
    """Seven balanced base-256 digits (most significant first, int64 arrays of
    y's shape) of trunc(y 2^(55 - E)), E = emax - 1022; |digit| <= 128."""
    t = np.trunc(np.ldexp(np.asarray(y, dtype=np.float64), 1077 - int(emax))).astype(np.int64)
    z = t + sum(128 << (8 * k) for k in range(7))
    d = [((z >> (8 * k)) & 0xFF) - 128 for k in range(6)] + [(z >> 48) - 128]
    return d[::-1]


def gram_tc_model(Y, sms):
    """G = Y^T Y as the tensor-core kernel forms it for Y (w x n): per CTA b of
    min(ceil(n/1024), sms) the chunks b, b + parts, ... of 1024 rows; exact
    integer sums hi (levels <= 3, weight 256^(3 - L)) and lo (levels 4..7,
    256^(7 - L)); the CTA's partial 2^(E_a + E_b - 14) (hi 2^-24 + lo 2^-56) in
    FP64; then the partials summed by four interleaved accumulators,
    (s0 + s1) + (s2 + s3), s_t over the CTAs c = t (mod 4) in order."""
    w, n = Y.shape
    emax = [int(bexp(Y[a]).max()) for a in range(w)]
    dig = np.stack([np.stack(digits55(Y[a], emax[a])) for a in range(w)], axis=1)  # [7][w][n]
    chunks = -(-n // 1024)
    parts = min(chunks, sms)
    partials = []
    for b in range(parts):
        rows = np.concatenate([np.arange(c * 1024, min(n, (c + 1) * 1024)) for c in range(b, chunks, parts)])
        D = dig[:, :, rows].astype(np.float64)
        hi = np.zeros((w, w), dtype=object)
        lo = np.zeros((w, w), dtype=object)
        for i in range(7):
            for j in range(min(7, LEVELS - i + 1)):
                L = i + j
                P = (D[i] @ D[j].T).astype(np.int64).astype(object)  # exact: |sum| < 2^53
                if L <= 3:
                    hi += P * 256 ** (3 - L)
                else:
                    lo += P * 256 ** (7 - L)
        part = np.empty((w, w))
        for a in range(w):
            for c in range(w):
                if emax[a] == 0x7FF or emax[c] == 0x7FF:
                    part[a, c] = math.nan
                    continue
                s = math.ldexp(float(hi[a, c]), -24) + math.ldexp(float(lo[a, c]), -56)
                part[a, c] = math.ldexp(s, emax[a] + emax[c] - 2058)
        partials.append(part)
    acc = [np.zeros((w, w)) for _ in range(4)]
    for c, part in enumerate(partials):
        acc[c % 4] = acc[c % 4] + part
    return (acc[0] + acc[1]) + (acc[2] + acc[3])


def recover_tc_model(Y, cf, x):
    """x + Y x', Y r', Y p' as the tensor-core recovery forms them (Y w x n,
    cf = [x', r', p']): Y's columns in 55-bit fixed point as above; the scaled
    coefficients u_vj = c_vj 2^(E_j - 55) in 55-bit fixed point under each
    vector's largest exponent F_v; digit products of levels d + e <= 7 summed
    exactly; one rounding to FP64 of T = T_hi 2^32 + T_lo times 2^(F_v - 15)."""
    w, n = Y.shape
    emax = [int(bexp(Y[j]).max()) for j in range(w)]
    yd = np.stack([np.stack(digits55(Y[j], emax[j])) for j in range(w)], axis=1).astype(np.float64)  # [7][w][n]
    outs = []
    for v in range(3):
        u = np.array([0.0 if emax[j] == 0 else math.ldexp(float(cf[v * w + j]), emax[j] - 1077) for j in range(w)])
        fv = int(bexp(u).max())
        ud = np.stack(digits55(u, fv)).astype(np.float64)  # [7][w]
        hi = np.zeros(n, dtype=object)
        lo = np.zeros(n, dtype=object)
        for L in range(LEVELS + 1):
            DL = np.zeros(n)
            for d in range(max(0, L - 6), min(6, L) + 1):
                DL += ud[L - d] @ yd[d]  # exact: |sum| < 2^22
            DL = DL.astype(np.int64).astype(object)
            if L <= 3:
                hi += DL * 256 ** (3 - L)
            else:
                lo += DL * 256 ** (7 - L)
        col = np.array([float(h * 2 ** 32 + l) for h, l in zip(hi, lo)]) * 2.0 ** (fv - 1037)
        outs.append(col)
    return x + outs[0], outs[1], outs[2]
