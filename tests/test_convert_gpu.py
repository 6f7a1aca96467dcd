"""FP64 <-> FP32 conversions done with integer operations on the IEEE 754 formats (complex
conversion, double-single split): bit-identical to the hardware / numpy round-to-nearest-even
conversions over the whole exponent range, ties, signed zeros, subnormals, overflow, inf and NaN."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _doubles(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) * 2.0 ** rng.integers(-160, 140, n)
    # exact ties between neighbouring floats (both parities of the last float bit)
    f = (rng.standard_normal(n // 4) * 2.0 ** rng.integers(-100, 100, n // 4)).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    ties = (f.astype(np.float64) + g.astype(np.float64)) / 2
    fmax = float(np.finfo(np.float32).max)
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-320, -1e-320, 2.0 ** -149, 2.0 ** -150,
                         2.0 ** -126, 2.0 ** -127, fmax, -fmax, fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -23),
                         1.0, -1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1e300, -1e-300])
    return np.concatenate([v, ties, specials])


def test_complex128_to_complex64_bitwise():
    import paper_1801_01473_gb300 as p
    d = _doubles(1 << 16, 11)
    z = torch.from_numpy((d[: len(d) // 2 * 2].reshape(-1, 2) @ np.array([1.0, 1j]))).cuda()
    ours = p.complex_convert(z, torch.complex64)
    ref = z.to(torch.complex64)
    assert torch.equal(torch.view_as_real(ours).view(torch.int32), torch.view_as_real(ref).view(torch.int32))


def test_complex64_to_complex128_bitwise():
    import paper_1801_01473_gb300 as p
    rng = np.random.default_rng(12)
    bits = rng.integers(0, 2 ** 32, 1 << 16, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    f = np.concatenate([f, np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, 1.0], dtype=np.float32)])
    f = f[: len(f) // 2 * 2]
    z = torch.from_numpy(f.view(np.complex64).copy()).cuda()
    ours = p.complex_convert(z, torch.complex128)
    ref = z.to(torch.complex128)
    a = torch.view_as_real(ours).view(torch.int64)
    b = torch.view_as_real(ref).view(torch.int64)
    nan = torch.isnan(torch.view_as_real(ref))
    assert torch.equal(a[~nan], b[~nan]) and bool(torch.isnan(torch.view_as_real(ours))[nan].all())


def test_double_single_split_bitwise():
    """pack to double-single: hi = RN32(d), lo = RN32(d - hi) for every value."""
    import paper_1801_01473_gb300 as p
    dims = (8, 8, 8, 8)
    lat = p.Lattice(dims)
    d = _doubles(4 * lat.Vh * 3, 13)
    d = d[np.isfinite(d)][: 2 * lat.Vh * 3]
    canon = (d[0::2] + 1j * d[1::2]).reshape(lat.Vh, 3)
    ds = p.pack(lat, torch.from_numpy(canon).cuda(), "ds").cpu().numpy().reshape(3, lat.Vh, 4)
    for part, col in (("re", (0, 1)), ("im", (2, 3))):
        x = (canon.real if part == "re" else canon.imag).T  # [3, Vh]
        with np.errstate(over="ignore", invalid="ignore"):
            hi = x.astype(np.float32)
            lo = (x - hi.astype(np.float64)).astype(np.float32)
        fin = np.isfinite(hi)
        np.testing.assert_array_equal(ds[..., col[0]][fin].view(np.uint32), hi[fin].view(np.uint32))
        np.testing.assert_array_equal(ds[..., col[1]][fin].view(np.uint32), lo[fin].view(np.uint32))
