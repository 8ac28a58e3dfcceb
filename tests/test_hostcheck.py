"""The kernels' step math compiled for the host (same header) against
independent references: scipy's Bessel functions and the FP64 oracle's Green's
function, radial CDF and inverse CDF (Supplemental 1.1), Philox known answers."""
import ctypes as C

import numpy as np
import pytest
import scipy.special as sp

DP = C.POINTER(C.c_double)


@pytest.fixture(scope="module")
def hc():
    from paper_2201_13240_gb300 import build as B
    return C.CDLL(B.build_hostcheck())


def _call(fn, *args, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    fn(*args, x.ctypes.data_as(DP), len(x), out.ctypes.data_as(DP))
    return out


X = np.concatenate([np.linspace(1e-3, 4, 300), np.linspace(4, 600, 300)])


@pytest.mark.parametrize("which", range(4))
def test_bessel_fp32_abramowitz_stegun(hc, which):
    ref = [sp.i0, sp.i1, sp.k0, sp.k1][which]
    x = X[X < 80]
    got = _call(hc.wos_hc_bessel_f32, which, x=x)
    assert np.max(np.abs(got / ref(x) - 1)) < 1e-5


@pytest.mark.parametrize("which", range(4))
def test_bessel_fp64(hc, which):
    ref = [sp.i0e, sp.i1e, sp.k0e, sp.k1e][which]
    scale = [np.exp(-X), np.exp(-X), np.exp(X), np.exp(X)][which]
    got = _call(hc.wos_hc_bessel_f64, which, x=X)
    assert np.max(np.abs(got * scale / ref(X) - 1)) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fp64", [0, 1])
def test_green_norm(hc, orc, dim, fp64):
    a = np.concatenate([[0.0], np.logspace(-4, 2.5, 200)])
    want = np.array([orc.green_norm(dim, 1.0, x * x) if x > 0 else 1 / (2 * dim) for x in a])
    got = _call(hc.wos_hc_green_q, dim, fp64, x=a)
    assert np.max(np.abs(got / want - 1)) < (1e-13 if fp64 else 5e-6)


A = [1e-4, 0.1, 0.5, 0.99, 1.0, 1.5, 1.99, 2.0, 2.5, 3.7, 3.8, 6.0, 20.0, 60.0, 200.0]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fp64", [0, 1])
def test_radial_cdf(hc, orc, dim, fp64):
    rho = np.linspace(1e-4, 1 - 1e-4, 120)
    for a in A:
        F = np.zeros_like(rho)
        P = np.zeros_like(rho)
        hc.wos_hc_radial(dim, fp64, C.c_double(a), rho.ctypes.data_as(DP), len(rho), F.ctypes.data_as(DP),
                         P.ctypes.data_as(DP))
        Fo = np.array([orc.green_cdf(dim, 1.0, a * a, r) for r in rho])
        Po = np.array([orc.green_pdf(dim, 1.0, a * a, r) for r in rho])
        assert np.max(np.abs(F - Fo)) < (1e-13 if fp64 else 2e-6), a
        assert np.max(np.abs(P - Po)) / np.max(np.abs(Po)) < (1e-12 if fp64 else 5e-6), a


@pytest.mark.parametrize("fp64", [0, 1])
def test_radial3_limits(hc, fp64):
    """The 3D radial law's two limits, each a closed form: a -> 0 gives the Beta(2,2) law
    F = 3 rho^2 - 2 rho^3 (density ~ rho (1 - rho)); large a gives the Gamma(2) law
    1 - F = e^{-x} (1 + x), x = a rho, up to e^{-a} terms (density ~ rho e^{-a rho})."""
    rho = np.concatenate([np.linspace(1e-6, 1 - 1e-6, 301), [1e-9, 1 - 1e-9]])
    tol = 1e-14 if fp64 else 3e-7

    def run(a):
        F = np.zeros_like(rho)
        P = np.zeros_like(rho)
        hc.wos_hc_radial(3, fp64, C.c_double(a), rho.ctypes.data_as(DP), len(rho), F.ctypes.data_as(DP),
                         P.ctypes.data_as(DP))
        return F, P

    for a in [0.0, 1e-30, 1e-9]:
        F, P = run(a)
        assert np.max(np.abs(F - (3 * rho ** 2 - 2 * rho ** 3))) < tol, a
        assert np.max(np.abs(P - 6 * rho * (1 - rho))) < 4 * tol, a
    for a in [150.0, 1000.0, 5000.0]:
        F, P = run(a)
        x = a * rho
        assert np.all(np.isfinite(F)) and np.all(np.isfinite(P)), a
        assert np.max(np.abs(F - (1 - np.exp(-x) * (1 + x)))) < tol, a
        want_p = a * x * np.exp(-x)
        assert np.max(np.abs(P - want_p)) / np.max(want_p) < 4 * tol, a


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fp64", [0, 1])
def test_sampled_radius_inverts_cdf(hc, orc, dim, fp64):
    for a in [1e-4, 0.3, 0.99, 1.01, 1.99, 2.01, 3.0, 5.0, 10.0, 30.0, 100.0, 400.0]:
        u = np.concatenate([np.linspace(1e-6, 1 - 1e-6, 200), [1e-7, 1e-5, 0.999999]])
        if not fp64:
            u = (np.floor(u * 2 ** 24) + 0.5) / 2 ** 24
        rho = np.zeros_like(u)
        hc.wos_hc_sample_radius(dim, fp64, C.c_double(a), u.ctypes.data_as(DP), len(u), rho.ctypes.data_as(DP))
        Fo = np.array([orc.green_cdf(dim, 1.0, a * a, r) for r in rho])
        # FP32: the sampled distribution's CDF is off by < 2e-6 (absolute)
        assert np.max(np.abs(Fo - u)) < (1e-12 if fp64 else 2e-6), a
        if fp64:
            ro = np.array([orc.green_inv(dim, 1.0, a * a, x) for x in u])
            assert np.max(np.abs(ro - rho)) < 1e-10, a


def test_philox_matches_oracle(hc, orc):
    rng = np.random.default_rng(0)
    for _ in range(50):
        ctr = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
        out = np.zeros(4, dtype=np.uint32)
        hc.wos_hc_philox(ctr.ctypes.data_as(C.POINTER(C.c_uint32)), key.ctypes.data_as(C.POINTER(C.c_uint32)),
                         out.ctypes.data_as(C.POINTER(C.c_uint32)))
        assert list(out) == orc.philox4x32_10(ctr, key)
        # the walk kernels' form with the round keys precomputed from the seed
        out_rk = np.zeros(4, dtype=np.uint32)
        hc.wos_hc_philox_rk(ctr.ctypes.data_as(C.POINTER(C.c_uint32)), key.ctypes.data_as(C.POINTER(C.c_uint32)),
                            out_rk.ctypes.data_as(C.POINTER(C.c_uint32)))
        assert list(out_rk) == list(out)


@pytest.mark.parametrize("dim", [2, 3])
def test_table_started_sampler(hc, orc, dim):
    """The FP32 sampler as the kernels run it (Newton from the FP64-built inverse-CDF
    table): its CDF error stays below 2e-6 and no warp needs more than a few iterations."""
    DPp = C.POINTER(C.c_double)
    for a in [1e-3, 0.5, 1.0, 2.0, 3.5, 7.0, 15.0, 31.0, 45.0]:
        u = (np.floor(np.random.default_rng(1).uniform(size=2048) * 2 ** 24) + 0.5) / 2 ** 24
        rho = np.zeros_like(u)
        it = np.zeros_like(u)
        hc.wos_hc_sample_f32(dim, 1, C.c_double(a), u.ctypes.data_as(DPp), len(u), rho.ctypes.data_as(DPp),
                             it.ctypes.data_as(DPp))
        Fo = np.array([orc.green_cdf(dim, 1.0, a * a, r) for r in rho[:400]])
        assert np.max(np.abs(Fo - u[:400])) < 2e-6, a
        if a < 32:
            assert it.reshape(-1, 32).max(axis=1).mean() <= 3.5, a


@pytest.mark.parametrize("dim", [2, 3])
def test_table_sampler_dense_scan(hc, orc, dim):
    """The FP32 sampler over the table's whole range (a < 32), including uniforms within
    1e-7 of 0 and 1: one Newton step from the table (or, in the last t interval, the
    safeguarded loop) leaves the exact CDF within 1.5e-6 of u."""
    DPp = C.POINTER(C.c_double)
    worst = 0.0
    for a in np.concatenate([np.linspace(0.0, 31.99, 97), [1e-6, 1e-3]]):
        rng = np.random.default_rng(int(a * 1000) + dim)
        u = np.concatenate([(np.floor(rng.uniform(size=240) * 2 ** 24) + 0.5) / 2 ** 24,
                            (np.arange(12) + 0.5) / 2 ** 24, 1.0 - (np.arange(12) + 0.5) / 2 ** 24])
        rho = np.zeros_like(u)
        it = np.zeros_like(u)
        hc.wos_hc_sample_f32(dim, 1, C.c_double(a), u.ctypes.data_as(DPp), len(u), rho.ctypes.data_as(DPp),
                             it.ctypes.data_as(DPp))
        assert np.all((rho > 0) & (rho < 1))
        Fo = np.array([orc.green_cdf(dim, 1.0, a * a, r) for r in rho])
        worst = max(worst, float(np.max(np.abs(Fo - u))))
        # inside the one-step range every lane does the same work
        inner = u < 1.0 - 2.0 / 512 ** 2
        assert np.all(it[inner] == 1)
    assert worst < 1.5e-6, worst


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fp64", [0, 1])
def test_centre_gradient_ratios(hc, orc, dim, fp64):
    """The kernels' grad G / G and grad P / P at the ball centre (Supplemental 1.3) against the
    oracle's printed forms, from the Laplace limit to large a.  FP32 cancels where G -> 0 at
    the sphere, so rho is kept at or below 0.9 for the tight bound."""
    R = 0.37
    rho = np.array([1e-4, 0.01, 0.1, 0.3, 0.5, 0.7, 0.9])
    tol = 1e-10 if fp64 else 1e-5
    for a in (0.0, 1e-5, 1e-3, 0.05, 0.3, 0.49, 0.51, 1.0, 1.9, 2.1, 3.0, 3.8, 10.0, 40.0, 150.0):
        out = np.zeros(2 * len(rho))
        hc.wos_hc_grad_ratios(dim, fp64, C.c_double(a), rho.ctypes.data_as(DP), len(rho), out.ctypes.data_as(DP))
        want = np.array([orc.green_grad_ratios(dim, R, (a / R) ** 2, r * R) for r in rho]) * R
        assert np.allclose(out.reshape(-1, 2), want, rtol=tol, atol=0), (a, out.reshape(-1, 2), want)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fp64", [0, 1])
def test_offcentre_kernels(hc, orc, dim, fp64):
    """The next-flight kernels' approximate off-centred G and P (Supplemental 1.2) against
    the oracle's, at random interior and sphere points, from the Laplace limit to a = 126."""
    rng = np.random.default_rng(0)
    tol = 1e-12 if fp64 else 1e-4
    for R, sb in ((0.3, 1e-3), (0.5, 4.0), (0.2, 787.0), (0.05, 1578.0), (1.0, 0.0), (0.4, 1e5)):
        n = 100

        def dirs():
            d = rng.normal(size=(n, 3))
            if dim == 2:
                d[:, 2] = 0
            return d / np.linalg.norm(d, axis=1)[:, None]
        u = dirs() * (R * rng.uniform(size=n) ** (1 / dim))[:, None]
        v = dirs() * (R * rng.uniform(size=n) ** (1 / dim))[:, None]
        z = dirs() * R
        out = np.zeros(2 * n)
        hc.wos_hc_offcentre(dim, fp64, C.c_double(R), C.c_double(sb), np.ascontiguousarray(u).ctypes.data_as(DP),
                            np.ascontiguousarray(v).ctypes.data_as(DP), np.ascontiguousarray(z).ctypes.data_as(DP),
                            n, out.ctypes.data_as(DP))
        scale = orc.green_G(dim, R, max(sb, 1e-12), 0.5 * R)
        for i in range(n):
            g = orc.offcentre_G(dim, R, sb, u[i, :dim], v[i, :dim])
            p = orc.offcentre_P(dim, R, sb, u[i, :dim], z[i, :dim])
            assert abs(out[2 * i] - g) <= tol * max(abs(g), scale), (R, sb, i)
            if abs(p) > 1e-30:
                assert abs(out[2 * i + 1] - p) <= tol * abs(p), (R, sb, i)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fp64", [0, 1])
@pytest.mark.parametrize("N", [1, 8, 32, 64])
def test_series_offcentre_kernels(hc, orc, dim, fp64, N):
    """The next-flight kernels' series G and P (Supplemental 1.2, N terms: ratio recurrences,
    Clenshaw sums) against the oracle's (power series, log-scaled), at random interior and
    sphere points including the ball centre, from a = 1e-3 to a = 100."""
    rng = np.random.default_rng(N)
    hc.wos_hc_nf_series.restype = C.c_int
    for R, sb in ((0.3, 1e-5), (0.5, 45.0), (0.2, 787.0), (1.0, 4.0), (0.1, 1e6)):
        n = 40

        def dirs():
            d = rng.normal(size=(n, 3))
            if dim == 2:
                d[:, 2] = 0
            return d / np.linalg.norm(d, axis=1)[:, None]
        u = dirs() * (R * rng.uniform(size=n) ** (1 / dim))[:, None]
        v = dirs() * (R * rng.uniform(size=n) ** (1 / dim))[:, None]
        z = dirs() * R
        u[0] = 0.0
        out = np.zeros(2 * n)
        rc = hc.wos_hc_nf_series(dim, fp64, C.c_double(R), C.c_double(sb), N,
                                 np.ascontiguousarray(u).ctypes.data_as(DP), np.ascontiguousarray(v).ctypes.data_as(DP),
                                 np.ascontiguousarray(z).ctypes.data_as(DP), n, out.ctypes.data_as(DP))
        assert rc == 0
        g = np.array([orc.series_G(dim, R, sb, u[i, :dim], v[i, :dim], N) for i in range(n)])
        p = np.array([orc.series_P(dim, R, sb, v[i, :dim], z[i, :dim], N) for i in range(n)])
        # G near the sphere is a difference of two larger terms: errors relative to the kernel's scale
        gs, ps = np.abs(g).max(), np.abs(p).max()
        tol = 1e-10 if fp64 else 2e-3
        assert np.all(np.abs(out[0::2] - g) <= tol * np.maximum(np.abs(g), 1e-2 * gs)), (R, sb)
        assert np.all(np.abs(out[1::2] - p) <= tol * np.maximum(np.abs(p), 1e-2 * ps)), (R, sb)
    bad = np.zeros(2)
    z3 = np.zeros(3)
    assert hc.wos_hc_nf_series(dim, fp64, C.c_double(1.0), C.c_double(1.0), 65, z3.ctypes.data_as(DP),
                               z3.ctypes.data_as(DP), z3.ctypes.data_as(DP), 1, bad.ctypes.data_as(DP)) == -1


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fp64", [0, 1])
def test_series_walk_sampling(hc, orc, dim, fp64):
    """The series walk's in-ball distance (h and its inverse, reading R24) against the oracle."""
    hc.wos_hc_nf_free.restype = C.c_int
    t = np.array([1e-6, 1e-3, 0.2, 0.499, 0.501, 1.0, 1.999, 2.001, 5.0, 30.0])
    out = np.zeros_like(t)
    hc.wos_hc_nf_free(dim, fp64, 0, C.c_double(0.0), C.c_double(0.0), t.ctypes.data_as(DP), len(t),
                      out.ctypes.data_as(DP))
    want = np.array([orc.nf_h(dim, x) for x in t])
    assert np.allclose(out, want, rtol=1e-13 if fp64 else 3e-6, atol=0), (out, want)
    u = np.array([1e-7, 1e-3, 0.1, 0.5, 0.9, 0.999])
    for sb, rm in ((45.0, 0.3), (4.0, 0.8), (900.0, 0.5), (1e-4, 0.2)):
        out = np.zeros_like(u)
        hc.wos_hc_nf_free(dim, fp64, 1, C.c_double(sb), C.c_double(rm), u.ctypes.data_as(DP), len(u),
                          out.ctypes.data_as(DP))
        want = np.array([orc.nf_free_radius(dim, sb, rm, x) for x in u])
        assert np.allclose(out, want, rtol=1e-12 if fp64 else 2e-5, atol=0), (sb, rm, out, want)


@pytest.mark.parametrize("fp64", [0, 1])
def test_uniforms21_equal_the_oracle(hc, orc, fp64):
    """The 3D step's six 21-bit uniforms (split and conversion) equal the oracle's exactly, in
    both precisions (the FP32 and FP64 walks draw identical values)."""
    rng = np.random.default_rng(3)
    w = rng.integers(0, 2 ** 32, size=(500, 4), dtype=np.uint64).astype(np.uint32)
    w[0] = 0
    w[1] = 0xFFFFFFFF
    out = np.zeros(6 * len(w))
    hc.wos_hc_uniforms21(fp64, np.ascontiguousarray(w).ctypes.data_as(C.POINTER(C.c_uint32)), len(w),
                         out.ctypes.data_as(DP))
    want = np.array([orc.uniforms21(x) for x in w]).ravel()
    assert np.array_equal(out, want)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fp64", [0, 1])
def test_green_log_derivative(hc, orc, dim, fp64):
    """R |G'/G| of the centred Green's function (the extra-drift weight) against the oracle."""
    R = 0.37
    rho = np.array([0.01, 0.1, 0.3, 0.5, 0.7, 0.9, 0.97])
    tol = 1e-10 if fp64 else 2e-5
    for a in (0.0, 1e-5, 1e-3, 0.05, 0.3, 1.0, 2.5, 8.0, 30.0):
        out = np.zeros(len(rho))
        hc.wos_hc_green_dlog(dim, fp64, C.c_double(a), rho.ctypes.data_as(DP), len(rho), out.ctypes.data_as(DP))
        want = np.array([orc.green_dlog(dim, R, (a / R) ** 2, r * R) for r in rho]) * R
        assert np.allclose(out, want, rtol=tol, atol=0), (a, out, want)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("lam", [0.97, 0.5])
def test_mixture_sample_matches_oracle(hc, orc, dim, lam):
    """The kernels' mixture ball sample (reading R22) equals the oracle's: FP64 radius and
    weight to rounding, FP32 within its sampler's tolerance."""
    R, sb = 0.35, 60.0
    a = np.sqrt(sb) * R
    u = np.ascontiguousarray(np.concatenate([np.linspace(0.001, 0.999, 401), [1e-7, 0.5 - 1e-9, lam, 1 - 1e-7]]))
    for fp64 in (1, 0):
        out = np.zeros(2 * len(u))
        hc.wos_hc_mix_radius(dim, fp64, C.c_double(a), C.c_double(lam), u.ctypes.data_as(DP), len(u),
                             out.ctypes.data_as(DP))
        for i, x in enumerate(u):
            r, w = orc.mix_radius(dim, R, sb, float(x), lam)
            if fp64:
                # the radius to rounding (in CDF terms where F is flat near rho = 1)
                r64 = out[2 * i] * R
                if x < lam:
                    assert abs(orc.green_cdf(dim, R, sb, r64) - x / lam) <= 1e-13
                    assert r64 == pytest.approx(r, rel=1e-7)
                else:
                    assert r64 == pytest.approx(r, rel=1e-13, abs=1e-15)
                # the weight at the radius drawn (the density vanishes like 1 - rho at the sphere)
                f = orc.green_pdf(dim, R, sb, r64) * R
                assert out[2 * i + 1] == pytest.approx(f / (lam * f + 1 - lam), rel=1e-8, abs=1e-13)
            else:
                # FP32: the radius within the sampler's CDF tolerance, the weight at that radius
                r32 = out[2 * i] * R
                if np.float32(x) < np.float32(lam):  # the branch as float32 compares it
                    assert abs(orc.green_cdf(dim, R, sb, r32) - float(np.float32(x)) / lam) <= 2e-6 or \
                        out[2 * i] >= 1.0 - 6e-8 - 1e-12  # clamped inside the uniform's resolution
                else:
                    # the uniform part in float32 arithmetic (u - lam cancels bits when lam ~ 1;
                    # the weight is taken at the radius actually drawn)
                    f32 = np.float32
                    want = (f32(x) - f32(lam)) / (f32(1) - f32(lam))
                    want = min(max(float(want), 1e-7), 1.0 - 6e-8)  # kept inside the uniform's resolution
                    assert out[2 * i] == pytest.approx(want, rel=1e-6, abs=1e-7)
                f = orc.green_pdf(dim, R, sb, r32) * R
                assert out[2 * i + 1] == pytest.approx(f / (lam * f + 1 - lam), rel=1e-4, abs=1e-5)


def test_fp32_uniform_from_bits(hc):
    """The FP32 uniform is ((x >> 9) + 1/2) 2^-23 exactly: inside (0, 1), symmetric about 1/2,
    and equal to the conversion formula it replaces."""
    x = np.concatenate([np.array([0, 1, 511, 512, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 513, 2 ** 32 - 1], dtype=np.uint64),
                        np.random.default_rng(3).integers(0, 2 ** 32, size=4096, dtype=np.uint64)]).astype(np.uint32)
    out = np.zeros(len(x))
    hc.wos_hc_uniform_f32(x.ctypes.data_as(C.POINTER(C.c_uint32)), len(x), out.ctypes.data_as(DP))
    want = ((x.astype(np.float64) // 512) + 0.5) / 2 ** 23
    assert np.array_equal(out, want)
    assert out.min() == 2.0 ** -24 and out.max() == 1 - 2.0 ** -24
