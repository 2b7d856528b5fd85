"""Shared helpers for the tests (no method arithmetic)."""
import numpy as np


def rel_err(a, r):
    """Tolerance metric: max_i |a_i - r_i| / (|r_i| + rms(r)).  Plain max relative error is
    ill-posed where a ReLU output is exactly zero, so each element's error is measured against
    its own magnitude plus the RMS of the whole reference."""
    a = np.asarray(a, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    if r.size == 0:
        return 0.0
    rms = float(np.sqrt(np.mean(r * r)))
    if rms == 0.0:
        return float(np.max(np.abs(a - r)))
    return float(np.max(np.abs(a - r) / (np.abs(r) + rms)))


FP32_TOL = 1e-4
BF16_TOL = 2e-2


def max_norm_err(a, r):
    """BF16 tolerance metric: max_i |a_i - r_i| / max_i |r_i|.  BF16 keeps 8 significant bits,
    so the absolute rounding error a layer adds scales with the magnitude of the values flowing
    through it rather than with each output's own size; near-zero outputs fed by large inputs
    make the per-element form (rel_err) exceed 2e-2 for an exact emulation of BF16 rounding."""
    a = np.asarray(a, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    if r.size == 0:
        return 0.0
    m = float(np.max(np.abs(r)))
    return float(np.max(np.abs(a - r))) / (m if m > 0 else 1.0)


def bf16_round(a):
    """Round to bfloat16 (nearest even) and back to float64, via torch's conversion."""
    import torch
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def bf16_emulated_backbone(canvas, conv_w, conv_bn, layers):
    """The oracle's backbone with every operand the BF16 path rounds rounded the same way:
    bf16 canvas, bf16 weights, bf16 layer outputs (FP64 accumulation in between)."""
    from oracle import pillars as O
    x = bf16_round(canvas)
    for (_ci, _co, s), w, bn in zip(layers, conv_w, conv_bn):
        x = bf16_round(O.conv3x3_bn_relu(x, bf16_round(w), bn, s))
    return x


def tf32_remainder(a):
    """x - (x with its 13 low mantissa bits cleared), in float32 (exact): the part of x a TF32
    read drops, computed from the bit pattern on the host."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    hi = (a.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    return (a - hi).astype(np.float32)
