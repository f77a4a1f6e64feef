"""Reference forward/backward of the learned proposal's MLP
(16 -> 64 -> 64 -> 1, relu, squared loss).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Plain numpy in FP64.  With ``bf16=True`` it rounds at the same points as
the GPU kernels (X, W1, W2, H1 and the dA2 operand of the dH1 product are
BF16, round to nearest even); with ``bf16=False`` it is the textbook
network, which the tests pin with central finite differences.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 16, 64
SIZES = [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("w3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def round_bf16(a) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a) -> np.ndarray:
    """BF16 bit patterns (uint16) of round_bf16(a)."""
    return (round_bf16(a).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def unpack(p):
    out, o = {}, 0
    for name, shape in SIZES:
        size = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + size], dtype=np.float64).reshape(shape)
        o += size
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def loss_and_grad(p, x, y, bf16: bool = True):
    """(z, loss, packed gradient) for rows x [B,16], targets y [B]."""
    q = unpack(p)
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = r(x)
    W1, W2 = r(q["W1"]), r(q["W2"])
    a1 = x @ W1 + q["b1"]
    h1 = r(np.maximum(a1, 0.0))
    a2 = h1 @ W2 + q["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ q["w3"] + q["b3"][0]
    B = x.shape[0]
    res = z - y
    loss = float(np.mean(res * res))
    dz = 2.0 * res / B
    g = {"w3": h2.T @ dz, "b3": np.array([dz.sum()])}
    da2 = np.outer(dz, q["w3"]) * (a2 > 0)
    g["W2"] = h1.T @ da2
    g["b2"] = da2.sum(axis=0)
    dh1 = r(da2) @ W2.T
    da1 = dh1 * (a1 > 0)
    g["W1"] = x.T @ da1
    g["b1"] = da1.sum(axis=0)
    return z, loss, pack(g)
