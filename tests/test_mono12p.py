"""Host side of the 12-bit packed input (Mono12p): the packer against the format's definition.

Mono12p (GenICam PFNC): pixel i of a frame occupies bits [12 i, 12 i + 12) of the frame's bytes
read as one little-endian bit string. The checks here use the definition directly: a worked
example written out by hand, and an unpacker that reads the bit string bit by bit
(numpy.unpackbits, little-endian bit order), which shares nothing with the packer's byte
arithmetic."""
import numpy as np
import pytest

import paper_2004_00923_b300 as dh


def _unpack_by_bits(packed: np.ndarray, npix: int) -> np.ndarray:
    bits = np.unpackbits(packed, axis=-1, bitorder="little")  # [F, 12 npix]
    bits = bits.reshape(packed.shape[0], npix, 12).astype(np.uint16)
    return (bits << np.arange(12, dtype=np.uint16)).sum(axis=-1).astype(np.uint16)


def test_worked_example():
    # pixels 0x123, 0xABC -> bit string 0xABC123 -> bytes 23 C1 AB; 0xFFF, 0x000 -> FF 0F 00
    f = np.array([[[0x123, 0xABC, 0xFFF, 0x000]]], dtype=np.uint16)
    assert dh.pack_mono12p(f).numpy().tolist() == [[0x23, 0xC1, 0xAB, 0xFF, 0x0F, 0x00]]


@pytest.mark.parametrize("shape", [(1, 2, 2), (3, 16, 16), (2, 64, 128)])
def test_round_trip_through_the_bit_string(shape):
    rng = np.random.default_rng(7)
    f = rng.integers(0, 4096, size=shape, dtype=np.uint16)
    p = dh.pack_mono12p(f).numpy()
    assert p.shape == (shape[0], shape[1] * shape[2] * 3 // 2) and p.dtype == np.uint8
    assert np.array_equal(_unpack_by_bits(p, shape[1] * shape[2]), f.reshape(shape[0], -1))


def test_rejects_values_beyond_12_bits_and_bad_shapes():
    with pytest.raises(ValueError):
        dh.pack_mono12p(np.full((1, 2, 2), 4096, dtype=np.uint16))
    with pytest.raises(TypeError):
        dh.pack_mono12p(np.zeros((1, 3, 1), dtype=np.uint16))  # odd pixel count
    with pytest.raises(TypeError):
        dh.pack_mono12p(np.zeros((1, 2, 2), dtype=np.int32))
