"""Reduced-precision snapshot storage, restated for the oracle (TEST INFRASTRUCTURE ONLY).

Form of the 16-bit storage: per field f, a scale s_f = max |v_f| over all cells
and snapshots (1 if the field is zero everywhere); each value is stored as the
round-to-nearest-even 16-bit float (bfloat16 or IEEE half) of the FP32 quotient
v_f / s_f; the value used by the transport is the stored value times s_f.

`quantize` returns the scale header, the stored records and the decoded FP32
array the oracle evaluates (stored value times scale, rounded to FP32), plus the
exact byte image of the device array, which the GPU quantizer must reproduce bit
for bit.
"""
import numpy as np

NFIELD = 18
HREC = 32
HHDR = 32


def _bf16_bits(q):
    """Round-to-nearest-even FP32 -> bfloat16 bit patterns (finite inputs)."""
    u = q.astype(np.float32).view(np.uint32)
    lsb = (u >> np.uint32(16)) & np.uint32(1)
    return ((u + np.uint32(0x7FFF) + lsb) >> np.uint32(16)).astype(np.uint16)


def _f16_bits(q):
    return q.astype(np.float32).astype(np.float16).view(np.uint16)


def _bits_to_f32(bits, dtype):
    if dtype == "bf16":
        return (bits.astype(np.uint32) << np.uint32(16)).view(np.float32)
    return bits.view(np.float16).astype(np.float32)


def quantize(fields, dtype):
    """fields: float32 [..., REC>=18] -> (header[32] f32, records[..., 32] u16, decoded[..., REC] f32, image u8)."""
    f = np.ascontiguousarray(fields, dtype=np.float32)
    vals = f[..., :NFIELD].reshape(-1, NFIELD)
    scale = np.abs(vals).max(axis=0).astype(np.float32)
    scale[scale == 0] = np.float32(1.0)
    q = (f[..., :NFIELD] / scale).astype(np.float32)          # FP32 quotient, correctly rounded
    bits = _bf16_bits(q) if dtype == "bf16" else _f16_bits(q)
    recs = np.zeros(f.shape[:-1] + (HREC,), dtype=np.uint16)
    recs[..., :NFIELD] = bits
    dec = np.zeros_like(f)
    dec[..., :NFIELD] = (_bits_to_f32(bits, dtype) * scale).astype(np.float32)
    header = np.zeros(HHDR, dtype=np.float32)
    header[:NFIELD] = scale
    image = np.concatenate([header.view(np.uint8), recs.reshape(-1).view(np.uint8)])
    return header, recs, dec, image
