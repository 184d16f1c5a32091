"""Pins of the oracle's 16-bit snapshot storage against library conversions.

torch's CPU float -> bfloat16 / float16 conversions (round to nearest even) are
independent implementations of the rounding the storage form specifies.
"""
import numpy as np
import pytest
import torch

from fte_inputs import configs
from oracle.quantize import quantize, NFIELD


@pytest.fixture(scope="module")
def fields():
    w = configs.scaled(configs.cir_uniform_1e6(), nr=64, nth=12, nph=36, n_snap=2)
    return configs.build_background(w)


@pytest.mark.parametrize("dtype,tdt", [("bf16", torch.bfloat16), ("f16", torch.float16)])
def test_rounding_matches_torch(fields, dtype, tdt):
    header, recs, dec, image = quantize(fields, dtype)
    scale = header[:NFIELD]
    q = torch.from_numpy((fields[..., :NFIELD] / scale).astype(np.float32))
    ref = q.to(tdt).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(recs[..., :NFIELD], ref)
    assert np.all(recs[..., NFIELD:] == 0)
    back = q.to(tdt).to(torch.float32).numpy() * scale
    assert np.array_equal(dec[..., :NFIELD], back.astype(np.float32))


def test_scales_and_error_bound(fields):
    header, recs, dec, image = quantize(fields, "bf16")
    vals = fields[..., :NFIELD].reshape(-1, NFIELD)
    assert np.array_equal(header[:NFIELD], np.abs(vals).max(axis=0))
    assert np.all(header[NFIELD:] == 0)
    # bfloat16 keeps 8 significant bits: relative rounding error <= 2^-8 (plus FP32 rounding)
    rel = np.abs(dec[..., :NFIELD] - fields[..., :NFIELD]) / np.maximum(np.abs(fields[..., :NFIELD]), 1e-30)
    assert rel.max() <= 2.0 ** -8 * (1 + 1e-6)
    # the byte image is the header followed by the records
    assert image.size == 32 * 4 + recs.size * 2
    assert np.array_equal(image[:128].view(np.float32), header)


def test_zero_field_gets_unit_scale():
    f = np.zeros((1, 2, 2, 2, 24), np.float32)
    f[..., 0] = 3.0
    header, recs, dec, _ = quantize(f, "f16")
    assert header[0] == 3.0 and np.all(header[1:NFIELD] == 1.0)
    assert np.all(dec[..., 0] == 3.0)
