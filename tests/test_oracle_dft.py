"""Pins of the oracle's DFT (Eq. eql_discrete2): brute-force sums, the library
FFT, Parseval, deltas and constants."""
import itertools

import numpy as np
import pytest

from oracle import dft

SHAPES = [(2, 3, 4), (3, 5, 2), (4, 4, 4), (5, 6, 3), (6, 2, 8), (12, 3, 16)]


def brute_forward(a):
    nz, ny, nx = a.shape[-3:]
    out = np.zeros(a.shape, dtype=complex)
    for kz, ky, kx in itertools.product(range(nz), range(ny), range(nx)):
        acc = 0j
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            ph = kz * z / nz + ky * y / ny + kx * x / nx
            acc = acc + a[..., z, y, x] * np.exp(-2j * np.pi * ph)
        out[..., kz, ky, kx] = acc / (nx * ny * nz)
    return out


@pytest.mark.parametrize("shape", SHAPES[:4])
def test_forward_matches_brute_force_sum(shape):
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2,) + shape)
    np.testing.assert_allclose(dft.forward(a), brute_forward(a), atol=1e-13, rtol=0)


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_library_fft(shape):
    rng = np.random.default_rng(2)
    a = rng.standard_normal((3,) + shape) + 1j * rng.standard_normal((3,) + shape)
    ref = np.fft.fftn(a, axes=(-3, -2, -1)) / np.prod(shape)
    np.testing.assert_allclose(dft.forward(a), ref, atol=1e-13, rtol=0)
    ref_inv = np.fft.ifftn(a, axes=(-3, -2, -1)) * np.prod(shape)
    np.testing.assert_allclose(dft.inverse(a), ref_inv, atol=1e-11, rtol=0)


@pytest.mark.parametrize("shape", SHAPES)
def test_roundtrip_and_parseval(shape):
    rng = np.random.default_rng(3)
    a = rng.standard_normal(shape)
    ahat = dft.forward(a)
    np.testing.assert_allclose(np.real(dft.inverse(ahat)), a, atol=1e-13)
    n = np.prod(shape)
    assert abs(np.sum(a * a) - n * np.sum(np.abs(ahat) ** 2)) < 1e-11 * np.sum(a * a)


def test_delta_and_constant():
    shape = (4, 6, 8)
    n = np.prod(shape)
    d = np.zeros(shape)
    d[0, 0, 0] = 1.0
    np.testing.assert_allclose(dft.forward(d), np.full(shape, 1.0 / n), atol=1e-16)
    c = np.full(shape, 2.5)
    chat = dft.forward(c)
    assert abs(chat[0, 0, 0] - 2.5) < 1e-14
    chat[0, 0, 0] = 0
    assert np.max(np.abs(chat)) < 1e-14
    # the null frequency of the 1/N-normalised transform is the voxel average
    rng = np.random.default_rng(4)
    a = rng.standard_normal(shape)
    assert abs(dft.forward(a)[0, 0, 0] - a.mean()) < 1e-15


def test_shifted_delta_is_pure_phase():
    shape = (4, 5, 6)
    d = np.zeros(shape)
    d[1, 2, 3] = 1.0
    nz, ny, nx = shape
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    expect = np.exp(-2j * np.pi * (kz * 1 / nz + ky * 2 / ny + kx * 3 / nx)) / d.size
    np.testing.assert_allclose(dft.forward(d), expect, atol=1e-15)


def test_signed_index_and_nyquist():
    assert list(dft.signed_index(6)) == [0, 1, 2, -3, -2, -1]
    assert list(dft.signed_index(5)) == [0, 1, 2, -2, -1]
    assert list(dft.nyquist_flag(6)) == [False, False, False, True, False, False]
    assert not dft.nyquist_flag(5).any()
