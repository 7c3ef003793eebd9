"""Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).

Stateless: every output block is a pure function of a 128-bit counter and a
64-bit key, so any element of any synthetic input can be regenerated on its
own, on the host here or on the device by the CUDA twin in
``synth/csrc/synth_gen.cu``.  Both follow the published definition:

* round:   (hi0, lo0) = mulhilo(0xD2511F53, c0); (hi1, lo1) = mulhilo(0xCD9E8D57, c2)
           c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
* key bump between rounds: k0 += 0x9E3779B9, k1 += 0xBB67AE85 (mod 2^32)
* ten rounds, the first one with the unbumped key.

This module draws random numbers only; it holds none of the solver's
arithmetic.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
_SH = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words for counters (c0, c1, c2, c3).

    Counters are broadcastable integer arrays (values < 2**32); the key words
    k0, k1 are Python ints.  Outputs are uint32 arrays of the broadcast shape.
    """
    shape = np.broadcast(np.asarray(c0), np.asarray(c1), np.asarray(c2), np.asarray(c3)).shape
    x0 = np.broadcast_to(np.asarray(c0, dtype=np.uint64), shape).copy()
    x1 = np.broadcast_to(np.asarray(c1, dtype=np.uint64), shape).copy()
    x2 = np.broadcast_to(np.asarray(c2, dtype=np.uint64), shape).copy()
    x3 = np.broadcast_to(np.asarray(c3, dtype=np.uint64), shape).copy()
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = x0 * _M0
        p1 = x2 * _M1
        hi0 = p0 >> _SH
        lo0 = p0 & _MASK
        hi1 = p1 >> _SH
        lo1 = p1 & _MASK
        y0 = hi1 ^ x1 ^ np.uint64(k0)
        y2 = hi0 ^ x3 ^ np.uint64(k1)
        x0, x1, x2, x3 = y0, lo1, y2, lo0
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return (x0.astype(np.uint32), x1.astype(np.uint32),
            x2.astype(np.uint32), x3.astype(np.uint32))


def complex_normal(c0, c1, c2, c3, seed):
    """Standard complex normal z (E|z|^2 = 1, Re and Im each N(0, 1/2)).

    Box-Muller on the first two output words of one Philox block:
    u1 = (w0 + 1/2) 2^-32, u2 = (w1 + 1/2) 2^-32, z = sqrt(-ln u1) exp(2 pi i u2).
    The key is (seed mod 2^32, seed >> 32).
    """
    w0, w1, _, _ = philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, seed >> 32)
    u1 = (w0.astype(np.float64) + 0.5) * (2.0 ** -32)
    u2 = (w1.astype(np.float64) + 0.5) * (2.0 ** -32)
    rho = np.sqrt(-np.log(u1))
    theta = (2.0 * np.pi) * u2
    return rho * np.cos(theta) + 1j * (rho * np.sin(theta))
