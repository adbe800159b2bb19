"""Parity of the preconditioner kernels (DST-I GEMM, partitioned tridiagonal solve, whole apply)
with the oracle, through the C ABI."""
import ctypes as C

import numpy as np
import pytest

from oracle import dst as odst
from oracle import precond as opre
from oracle.tridiag import thomas
from paper_1005_0542_gb300 import inputs
from paper_1005_0542_gb300 import lagwave as L

from gpu_util import make_ctx, dev, empty, host, medium, plan, plan_info, ptr, rel, torch

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(77)
TOL64 = 1e-12          # float64 kernels vs float64 oracle (rounding order only)
TOL_MIXED = 2e-4       # float32 preconditioner vs float64 oracle


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    L.lag_destroy(c)


@pytest.mark.parametrize("nx", [1, 2, 3, 5, 31, 64, 127, 200, 1024])
def test_dst_f64(ctx, nx):
    nz, nrhs = 7, 3
    x = RNG.standard_normal((nrhs, nz, nx))
    p = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1)
    xd, yd = dev(x), empty(x.shape)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(yd), nrhs), ctx)
    assert rel(host(yd), odst.dst_x(x)) < 1e-13
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("nz,nx", [(4, 3), (33, 17), (100, 64), (129, 130), (1024, 40)])
def test_tridiag_f64_every_partition_count(ctx, P, nz, nx):
    dx, dz, ax, az, d = 5.0, 3.0, 2.0e9, 1.5e9, 4.0e7
    p = plan(ctx, nx, nz, dx, dz, ax, az, d, partitions=P)
    Pgot, Lp, _ = plan_info(p)
    assert Pgot <= P and Pgot * Lp >= nz
    nrhs = 2
    rhs = RNG.standard_normal((nrhs, nz, nx))
    diag = opre.mode_diagonals(nx, dx, dz, ax, az, d)
    off = -az / dz ** 2
    ref = np.moveaxis(thomas(off, diag, off, np.moveaxis(rhs, 1, 0)), 0, 1)
    dd, yd = dev(rhs), empty(rhs.shape)
    L.check(L.lag_precond_tridiag(p, ptr(dd), ptr(yd), nrhs), ctx)
    assert rel(host(yd), ref) < 1e-13
    # in place gives the same bits
    L.check(L.lag_precond_tridiag(p, ptr(dd), ptr(dd), nrhs), ctx)
    assert np.array_equal(host(dd), host(yd))
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("nz,nx", [(16, 16), (33, 20), (128, 128), (257, 96)])
def test_precond_apply_f64(ctx, nz, nx):
    dx, dz, ax, az, d = 10.0, 7.0, 3.0e9, 3.0e9, 1.0e7
    p = plan(ctx, nx, nz, dx, dz, ax, az, d)
    r = RNG.standard_normal((3, nz, nx))
    rd, zd = dev(r), empty(r.shape)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 3), ctx)
    assert rel(host(zd), opre.apply_inverse(r, dx, dz, ax, az, d)) < TOL64
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("nz,nx", [(33, 20), (128, 128), (64, 1024)])
def test_tridiag_f32(ctx, nz, nx):
    dx, dz, ax, az, d = 5.0, 5.0, 2.0e10, 2.0e10, 1.0e7
    p = plan(ctx, nx, nz, dx, dz, ax, az, d, prec=L.LAG_MIXED)
    t = torch()
    rhs = RNG.standard_normal((2, nz, nx)).astype(np.float32)
    diag = opre.mode_diagonals(nx, dx, dz, ax, az, d)
    off = -az / dz ** 2
    ref = np.moveaxis(thomas(off, diag, off, np.moveaxis(rhs.astype(np.float64), 1, 0)), 0, 1)
    dd = dev(rhs)
    yd = t.empty(rhs.shape, dtype=t.float32, device="cuda")
    L.check(L.lag_precond_tridiag_f32(p, ptr(dd), ptr(yd), 2), ctx)
    assert rel(host(yd), ref) < 2e-5
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("nz,nx", [(33, 20), (128, 128), (64, 1024), (32, 2048)])
def test_precond_apply_mixed(ctx, nz, nx):
    dx, dz, ax, az, d = 5.0, 5.0, 2.0e10, 2.0e10, 1.0e7
    p = plan(ctx, nx, nz, dx, dz, ax, az, d, prec=L.LAG_MIXED)
    r = RNG.standard_normal((2, nz, nx))
    rd, zd = dev(r), empty(r.shape)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 2), ctx)
    assert rel(host(zd), opre.apply_inverse(r, dx, dz, ax, az, d)) < TOL_MIXED
    L.lag_precond_destroy(p)


def test_precond_edge_cases(ctx):
    p = plan(ctx, 8, 8, 1.0, 1.0, 1.0, 1.0, 0.5)
    assert L.lag_precond_apply(p, None, None, 0) == L.LAG_OK          # empty batch
    assert L.lag_precond_apply(p, None, None, -1) == L.LAG_EINVAL
    assert L.lag_precond_apply(None, None, None, 1) == L.LAG_EINVAL
    q = C.c_void_p()
    g = L.grid(8, 8, 1.0, 1.0)
    assert L.lag_precond_create_sep(ctx, C.byref(g), -1.0, 1.0, 0.0, 0, 0, C.byref(q)) == L.LAG_EINVAL
    assert L.lag_precond_create_sep(ctx, C.byref(g), 1.0, 1.0, 0.0, 7, 0, C.byref(q)) == L.LAG_EINVAL
    assert L.lag_precond_tridiag_f32(p, None, None, 1) == L.LAG_EINVAL  # float32 solve needs a mixed plan
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("prec,tol", [(L.LAG_FP64, TOL64), (L.LAG_MIXED, TOL_MIXED)])
def test_precond_full_size_bench_config(ctx, prec, tol):
    # the standalone preconditioner workload: 1024 modes x nz = 1024 x 512 right-hand sides,
    # midrange coefficients of the 2048 x 1024 random layered model at 5 m; two sampled
    # right-hand sides are checked against the oracle one by one
    shot = inputs.random_layered(nx=2048, nz=1024, hx=5.0, n_harm=1)
    kap = shot.rho * shot.c ** 2
    ax, az, d = opre.acoustic_params(kap, shot.rho, shot.h)
    nx, nz, nrhs = 1024, 1024, 512
    p = plan(ctx, nx, nz, 5.0, 5.0, ax, az, d, prec=prec)
    t = torch()
    gen = t.Generator(device="cuda").manual_seed(5)
    rd = t.randn((nrhs, nz, nx), dtype=t.float64, device="cuda", generator=gen)
    zd = t.empty_like(rd)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), nrhs), ctx)
    for b in (0, 311):
        r = host(rd[b])
        assert rel(host(zd[b]), opre.apply_inverse(r, 5.0, 5.0, ax, az, d)) < tol
    L.lag_precond_destroy(p)
    del rd, zd
    t.cuda.empty_cache()


@pytest.mark.parametrize("products,tol", [(3, 5e-5), (2, 8e-3), (1, 1.5e-2)])
@pytest.mark.parametrize("nx", [16, 17, 64, 300, 1024, 2048])
def test_dst_tensor_cores_forward_and_inverse(ctx, nx, products, tol):
    # mixed plans run the DST on tcgen05 (bf16 products, FP32 accumulate): forward (float64 in,
    # float32 spectrum) and inverse (float32 spectrum in, float64 out) against the oracle; the
    # tolerance follows the operand rounding (split: 2^-16, S in bf16: 2^-9)
    nz, nrhs = 9, 3
    p = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1, prec=L.LAG_MIXED)
    assert L.lag_precond_uses_tensor_cores(p) == 1
    L.check(L.lag_precond_set_dst_products(p, products), ctx)
    x = RNG.standard_normal((nrhs, nz, nx))
    xd, yd = dev(x), empty(x.shape)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(yd), nrhs), ctx)
    ref = odst.dst_x(x)
    assert rel(host(yd), ref) < tol
    sf = dev(ref.astype(np.float32))
    zd = empty(x.shape)
    L.check(L.lag_precond_dst_f32(p, ptr(sf), ptr(zd), nrhs), ctx)
    assert rel(host(zd), odst.dst_x(ref.astype(np.float32).astype(np.float64))) < tol
    L.lag_precond_destroy(p)


def test_mixed_apply_simt_and_tensor_cores_agree(ctx, monkeypatch):
    nx, nz = 256, 64
    args = (nx, nz, 5.0, 5.0, 2.0e10, 2.0e10, 1.0e7)
    r = RNG.standard_normal((2, nz, nx))
    rd = dev(r)
    p_tc = plan(ctx, *args, prec=L.LAG_MIXED)
    monkeypatch.setenv("LAGWAVE_DST_KERNEL", "simt")
    p_simt = plan(ctx, *args, prec=L.LAG_MIXED)
    assert L.lag_precond_uses_tensor_cores(p_tc) == 1 and L.lag_precond_uses_tensor_cores(p_simt) == 0
    z1, z2 = empty(r.shape), empty(r.shape)
    L.check(L.lag_precond_apply(p_tc, ptr(rd), ptr(z1), 2), ctx)
    L.check(L.lag_precond_apply(p_simt, ptr(rd), ptr(z2), 2), ctx)
    ref = opre.apply_inverse(r, 5.0, 5.0, 2.0e10, 2.0e10, 1.0e7)
    assert rel(host(z1), ref) < TOL_MIXED and rel(host(z2), ref) < TOL_MIXED
    L.lag_precond_destroy(p_tc)
    L.lag_precond_destroy(p_simt)


def test_tensor_core_dst_many_tiles(ctx):
    # more tiles than SMs: the persistent kernel walks several tiles per CTA, alternating its two
    # tensor-memory accumulators
    nx, nz, nrhs = 1024, 256, 24           # 6144 rows -> 48 m tiles x 2 n tiles x 2 parities
    p = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1, prec=L.LAG_MIXED)
    x = RNG.standard_normal((nrhs, nz, nx))
    xd, yd = dev(x), empty(x.shape)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(yd), nrhs), ctx)
    assert rel(host(yd), odst.dst_x(x)) < 5e-5
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("products", [1, 2, 3])
def test_mixed_pcg_converges_with_every_product_count(ctx, products):
    # the flexible PCG reaches the float64 tolerance whatever the DST's bf16 product count
    from oracle import fd, krylov
    nz, nx, h, dx = 48, 80, 200.0, 5.0
    c = RNG.uniform(1500, 4500, (nz, nx))
    rho = 310 * c ** 0.25
    m = medium(ctx, nx, nz, dx, dx, c, rho, h)
    mid = (C.c_double * 3)()
    L.check(L.lag_medium_midranges(m, mid))
    p = plan(ctx, nx, nz, dx, dx, mid[0], mid[0], mid[1] * h * h / 4, prec=L.LAG_MIXED)
    L.check(L.lag_precond_set_dst_products(p, products), ctx)
    b = RNG.standard_normal((2, nz, nx))
    bd, xd = dev(b), empty(b.shape)
    its = (C.c_int * 2)()
    res = (C.c_double * 2)()
    s = L.solver(tol=1e-11, prec=L.LAG_MIXED)
    L.check(L.lag_solve_system(m, p, None, ptr(bd), ptr(xd), 2, C.byref(s), its, res), ctx)
    kap = fd.kappa_from_velocity(c, rho)
    x = host(xd)
    for i in range(2):
        r = b[i] - fd.apply_A(x[i], kap, rho, h, dx, dx)
        assert np.linalg.norm(r) / np.linalg.norm(b[i]) < 1e-10
    L.lag_precond_destroy(p)
    L.lag_medium_destroy(m)


def test_autotune_keeps_a_valid_preconditioner(ctx):
    nx, nz, nrhs = 512, 256, 4
    args = (nx, nz, 5.0, 5.0, 2.0e10, 2.0e10, 1.0e7)
    p = plan(ctx, *args, prec=L.LAG_MIXED)
    P, MT, K, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
    L.check(L.lag_precond_autotune(p, nrhs, C.byref(P), C.byref(MT), C.byref(K), C.byref(ms)), ctx)
    assert 1 <= P.value <= 32 and K.value in (1, 2, 3) and ms.value > 0
    assert plan_info(p)[0] == P.value and plan_info(p)[2] == MT.value
    r = RNG.standard_normal((2, nz, nx))
    rd, zd = dev(r), empty(r.shape)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 2), ctx)
    tol = TOL_MIXED if K.value == 3 else 2e-2
    assert rel(host(zd), opre.apply_inverse(r, *args[2:])) < tol
    L.lag_precond_destroy(p)
    q = plan(ctx, *args, prec=L.LAG_FP64)
    L.check(L.lag_precond_autotune(q, nrhs, C.byref(P), C.byref(MT), C.byref(K), C.byref(ms)), ctx)
    assert K.value == 3 and plan_info(q)[2] == MT.value
    L.check(L.lag_precond_apply(q, ptr(rd), ptr(zd), 2), ctx)
    assert rel(host(zd), opre.apply_inverse(r, *args[2:])) < TOL64
    L.lag_precond_destroy(q)


@pytest.mark.parametrize("prec", [L.LAG_FP64, L.LAG_MIXED])
def test_every_layout_of_the_tridiagonal_solve(ctx, prec):
    # every (partition count, mode tile) the register kernel offers solves the same systems
    # (ragged nx so the last mode tile is partial, ragged nz so the last partition is padded)
    nx, nz, nrhs = 75, 100, 3
    dx, dz, ax, az, d = 5.0, 4.0, 2.0e10, 1.5e10, 1.0e7
    p = plan(ctx, nx, nz, dx, dz, ax, az, d, prec=prec)
    f64 = prec == L.LAG_FP64
    tiles = (4, 8) if f64 else (8, 16, 32)
    rhs = RNG.standard_normal((nrhs, nz, nx))
    diag = opre.mode_diagonals(nx, dx, dz, ax, az, d)
    off = -az / dz ** 2
    ref = np.moveaxis(thomas(off, diag, off, np.moveaxis(rhs, 1, 0)), 0, 1)
    t = torch()
    seen = set()
    for parts in (4, 8, 16, 32):          # nz = 100: (P, L) = (4, 32), (7, 16), (13, 8), (25, 4)
        for mt in tiles:
            L.check(L.lag_precond_set_layout(p, parts, mt), ctx)
            P, Lp, got_mt = plan_info(p)
            assert got_mt == mt and P * Lp >= nz
            seen.add((P, mt))
            if f64:
                dd, yd = dev(rhs), empty(rhs.shape)
                L.check(L.lag_precond_tridiag(p, ptr(dd), ptr(yd), nrhs), ctx)
                assert rel(host(yd), ref) < 1e-13
            else:
                dd = dev(rhs.astype(np.float32))
                yd = t.empty(rhs.shape, dtype=t.float32, device="cuda")
                L.check(L.lag_precond_tridiag_f32(p, ptr(dd), ptr(yd), nrhs), ctx)
                assert rel(host(yd), ref) < 2e-5
    assert len(seen) == 4 * len(tiles)
    assert L.lag_precond_set_layout(p, 8, 12) == L.LAG_EINVAL     # not a tile of the kernel
    assert L.lag_precond_set_layout(p, 1, 8) == L.LAG_EINVAL      # L = 128: shared-memory kernel
    assert L.lag_precond_set_layout(p, 33, 0) == L.LAG_EINVAL     # more partitions than lanes
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("nx", [16, 17, 255, 2048, 4096])
def test_dst_f64_exact_slices_row_scales(ctx, nx):
    # the float64 DST on the tensor cores (exact bf16 slices, float64 sums): every row to float64
    # accuracy relative to its own size, whatever the rows' magnitudes; zero rows stay zero
    nz, nrhs = 8, 2
    x = RNG.standard_normal((nrhs, nz, nx))
    scales = 10.0 ** np.array([-306, -150, -8, 0, 3, 17, 150, 305])
    x = x * scales[None, :, None] / np.sqrt(nx)  # rows of any magnitude, near both ends of the range
    x[1, 2] = 0.0
    p = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1)
    assert L.lag_precond_uses_tensor_cores(p) == 1
    xd, yd = dev(x), empty(x.shape)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(yd), nrhs), ctx)
    y, ref = host(yd), odst.dst_x(x)
    sc = np.abs(ref).max(axis=-1, keepdims=True)           # per-row scale (norms of 1e305 rows overflow)
    sc = np.where(sc > 0, sc, 1.0)
    err = np.linalg.norm((y - ref) / sc, axis=-1) / np.maximum(np.linalg.norm(ref / sc, axis=-1), 1e-300)
    assert np.all(np.isfinite(y))
    assert err.max() < 1e-14
    assert np.all(y[1, 2] == 0.0)
    L.lag_precond_destroy(p)


def test_dst_f64_exact_slices_nonfinite_row(ctx):
    # a non-finite input row gives a non-finite output row and leaves the others exact
    nx, nz = 64, 4
    x = RNG.standard_normal((1, nz, nx))
    x[0, 1, 5] = np.nan
    p = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1)
    xd, yd = dev(x), empty(x.shape)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(yd), 1), ctx)
    y = host(yd)
    assert np.all(np.isnan(y[0, 1]))
    ok = [0, 2, 3]
    assert rel(y[0, ok], odst.dst_x(x[:, ok])[0]) < 1e-14
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("nx,nz,nrhs", [(16, 3, 1), (255, 130, 1), (2048, 1024, 1), (1000, 77, 5), (4096, 256, 2)])
def test_dst_f64_two_sm_pairs_equal_one_sm_tiles(ctx, monkeypatch, nx, nz, nrhs):
    # the exact-slice GEMM on two-SM pairs (cta_group::2: 256-row tile pairs, each SM holding half
    # of the B columns) against the one-SM kernel: the same exact slice products and int64 sums,
    # so the same float64 results; row counts that leave the last pair half empty, ragged columns
    x = RNG.standard_normal((nrhs, nz, nx))
    p = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1)
    assert L.lag_precond_uses_tensor_cores(p) == 1
    xd, y2, y1 = dev(x), empty(x.shape), empty(x.shape)
    assert L.lag_precond_dst_gemm(p, nrhs) == L.LAG_GEMM_SLICE_TILES
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(y1), nrhs), ctx)
    monkeypatch.setenv("LAGWAVE_OZ_PAIR", "1")
    assert L.lag_precond_dst_gemm(p, nrhs) == L.LAG_GEMM_SLICE_PAIRS
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(y2), nrhs), ctx)
    monkeypatch.delenv("LAGWAVE_OZ_PAIR")
    a, b = host(y2), host(y1)
    assert rel(a, b) < 1e-15
    assert rel(a, odst.dst_x(x)) < 1e-14
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("nx", [16, 255, 1000, 2048])
def test_dst_f64_eight_bit_slices_equal_seven_bit(ctx, monkeypatch, nx):
    # the 8-bit exact-slice format (28 pairs, exact pairs in K chunks of 256) against the 7-bit one
    # (36 pairs): two different exact decompositions of the same float64 products
    nz, nrhs = 40, 2
    x = RNG.standard_normal((nrhs, nz, nx)) * 10.0 ** RNG.uniform(-30, 30, (nrhs, nz, 1))
    p8 = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1)
    monkeypatch.setenv("LAGWAVE_OZ_BITS", "7")
    p7 = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1)
    monkeypatch.delenv("LAGWAVE_OZ_BITS")
    xd, y8, y7 = dev(x), empty(x.shape), empty(x.shape)
    L.check(L.lag_precond_dst(p8, ptr(xd), ptr(y8), nrhs), ctx)
    L.check(L.lag_precond_dst(p7, ptr(xd), ptr(y7), nrhs), ctx)
    a, b, ref = host(y8), host(y7), odst.dst_x(x)
    sc = np.abs(ref).max(axis=-1, keepdims=True)
    assert np.abs((a - ref) / sc).max() < 1e-14 and np.abs((b - ref) / sc).max() < 1e-14
    assert np.abs((a - b) / sc).max() < 1e-14
    L.lag_precond_destroy(p8)
    L.lag_precond_destroy(p7)


def _streamk_expected(nx, nz, nrhs):
    # the host's rule: one right-hand side, tiles not a multiple of the SM count, G/2 <= tiles < 4 G
    sms = torch().cuda.get_device_properties(0).multi_processor_count
    tiles = -(-nz // 128) * (-(-((nx + 1) // 2) // 128) + -(-(nx // 2) // 128))
    return nrhs == 1 and tiles % sms != 0 and 2 * tiles >= sms and tiles < 4 * sms


@pytest.mark.parametrize("nx,nz", [(2048, 1024), (2048, 640), (2000, 600), (2047, 700), (1024, 1536), (2560, 1280)])
def test_dst_f64_stream_k_matches_tiles_and_oracle(ctx, monkeypatch, nx, nz):
    # one right-hand side whose output tiles leave SMs idle in a last wave: the stream-K GEMM (the
    # steps of all tiles cut into one equal range per SM, a split tile finished from int64 parts by
    # the CTA holding its last step) against the tile kernel and the oracle's DST; ragged rows and
    # columns, an odd length, the 7-bit format (ceil(n/2) > 1024), rows scaled over 40 decades, a
    # non-finite row, and repeated launches (the ticket counters and epoch reset by the last CTA)
    x = RNG.standard_normal((1, nz, nx)) * 10.0 ** RNG.uniform(-20, 20, (1, nz, 1))
    x[0, nz // 3, nx // 2] = np.inf
    p = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1)
    assert L.lag_precond_dst_gemm(p, 1) == L.LAG_GEMM_SLICE_TILES  # stream-K is opt-in
    monkeypatch.setenv("LAGWAVE_OZ_SK", "1")
    if torch().cuda.get_device_properties(0).multi_processor_count == 152:
        assert _streamk_expected(nx, nz, 1)  # every case here splits tiles on a 152-SM GB300
    want = L.LAG_GEMM_SLICE_STREAMK if _streamk_expected(nx, nz, 1) else L.LAG_GEMM_SLICE_TILES
    assert L.lag_precond_dst_gemm(p, 1) == want
    assert L.lag_precond_dst_gemm(p, 2) == L.LAG_GEMM_SLICE_TILES
    xd, ys, yt = dev(x), empty(x.shape), empty(x.shape)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(ys), 1), ctx)
    first = host(ys)
    assert L.lag_precond_status(p) == L.LAG_OK
    for _ in range(3):
        ys.fill_(7.0)  # every output is written again
        L.check(L.lag_precond_dst(p, ptr(xd), ptr(ys), 1), ctx)
        assert np.array_equal(host(ys), first, equal_nan=True)
    monkeypatch.delenv("LAGWAVE_OZ_SK")
    assert L.lag_precond_dst_gemm(p, 1) == L.LAG_GEMM_SLICE_TILES
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(yt), 1), ctx)
    monkeypatch.setenv("LAGWAVE_OZ_SK", "1")
    a, b = first[0], host(yt)[0]
    bad = nz // 3
    assert np.all(np.isnan(a[bad])) and np.all(np.isnan(b[bad]))
    ok = np.arange(nz) != bad
    ref = odst.dst_x(x[:, ok])[0]
    sc = np.abs(ref).max(axis=-1, keepdims=True)
    assert np.abs((a[ok] - b[ok]) / sc).max() < 1e-15
    assert np.abs((a[ok] - ref) / sc).max() < 1e-14
    # the same transform inside a batch of two runs the tile kernel and gives the same rows
    x2 = np.concatenate([x, x[:, ::-1]], axis=0)
    x2d, y2 = dev(x2), empty(x2.shape)
    L.check(L.lag_precond_dst(p, ptr(x2d), ptr(y2), 2), ctx)
    assert np.abs((host(y2)[0][ok] - b[ok]) / sc).max() == 0.0
    # and stream-K again after the batch (its scratch regrown: counters and slots kept apart)
    ys.fill_(7.0)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(ys), 1), ctx)
    assert np.array_equal(host(ys), first, equal_nan=True)
    assert L.lag_precond_status(p) == L.LAG_OK
    monkeypatch.delenv("LAGWAVE_OZ_SK")
    L.lag_precond_destroy(p)


def test_dst_f64_tiles_stored_from_registers_and_by_the_whole_cta(ctx):
    # 3 x 1024 rows of 2048: 384 output tiles on at most 152 CTAs, so a CTA stores its earlier tiles
    # from the epilogue warps' registers and its last one through shared memory with all ten warps.
    # Both against the oracle's DST (rows over 40 decades, rows at 1e-300 and 3e304 whose results
    # leave the integer conversion's range, a non-finite row), and the first right-hand side
    # bit for bit against the same rows transformed alone (128 tiles: every tile a last tile)
    nx, nz, nrhs = 2048, 1024, 3
    x = RNG.standard_normal((nrhs, nz, nx)) * 10.0 ** RNG.uniform(-20, 20, (nrhs, nz, 1))
    x[0, 5] = RNG.standard_normal(nx) * 1e-300  # results normal, below the integer conversion's range
    x[1, 700] = RNG.standard_normal(nx) * 3e304  # and above it
    x[2, 300, 17] = np.nan
    p = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1)
    assert L.lag_precond_dst_gemm(p, nrhs) == L.LAG_GEMM_SLICE_TILES
    xd, y3, y1 = dev(x), empty(x.shape), empty(x[:1].shape)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(y3), nrhs), ctx)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(y1), 1), ctx)
    a = host(y3)
    assert np.array_equal(a[0], host(y1)[0])
    assert np.all(np.isnan(a[2, 300]))
    for b in range(nrhs):
        rows = np.arange(b, nz, 5)  # a sample of every 5th row of each right-hand side
        rows = np.union1d(rows, [5, 700])
        rows = rows[~((b == 2) & (rows == 300))]
        ref = odst.dst_x(x[b:b + 1, rows])[0]
        sc = np.abs(ref).max(axis=-1, keepdims=True)
        assert np.abs((a[b, rows] - ref) / sc).max() < 1e-14
    L.lag_precond_destroy(p)


def test_dst_gemm_query(ctx, monkeypatch):
    # the GEMM kernel a transform launches, by plan kind, right-hand sides and environment
    pm = plan(ctx, 2048, 1024, 5.0, 5.0, 1.0, 1.0, 0.1, prec=L.LAG_MIXED)
    assert L.lag_precond_dst_gemm(pm, 1) == L.LAG_GEMM_SPLIT_BF16
    assert L.lag_precond_dst_gemm(pm, 0) == L.LAG_EINVAL
    assert L.lag_precond_dst_gemm(None, 1) == L.LAG_EINVAL
    L.lag_precond_destroy(pm)
    p = plan(ctx, 64, 8, 5.0, 5.0, 1.0, 1.0, 0.1)  # 2 tiles: too few to split over the SMs
    assert L.lag_precond_dst_gemm(p, 1) == L.LAG_GEMM_SLICE_TILES
    L.lag_precond_destroy(p)
    monkeypatch.setenv("LAGWAVE_DST_KERNEL", "simt")
    ps = plan(ctx, 64, 8, 5.0, 5.0, 1.0, 1.0, 0.1)
    monkeypatch.delenv("LAGWAVE_DST_KERNEL")
    assert L.lag_precond_dst_gemm(ps, 1) == L.LAG_GEMM_SIMT
    L.lag_precond_destroy(ps)


@pytest.mark.parametrize("shape", ["2x2", "1x2", "2x1"])
@pytest.mark.parametrize("nx,nz,nrhs", [(2048, 1024, 1), (700, 130, 3), (16, 3, 1), (1000, 77, 5), (4096, 256, 2)])
def test_dst_f64_cluster_multicast_equals_tiles(ctx, monkeypatch, shape, nx, nz, nrhs):
    # tiles on clusters (2 x 2, 1 x 2, 2 x 1 tiles) whose shared A / B slice tiles are read from L2
    # once and multicast into every CTA that needs them, against the one-CTA tile kernel: the same
    # exact products; the FP32-rounded tail pairs are grouped by weight here and by A slice in the
    # tile kernel, so the two differ by those roundings only (far below the float64 rounding).  An
    # odd column-tile count (700: 3 column tiles per parity; 16: 1), padding m-tiles, batches, the
    # 6-bit format (4096), rows over 40 decades
    x = RNG.standard_normal((nrhs, nz, nx)) * 10.0 ** RNG.uniform(-20, 20, (nrhs, nz, 1))
    p = plan(ctx, nx, nz, 5.0, 5.0, 1.0, 1.0, 0.1)
    xd, yc, yt = dev(x), empty(x.shape), empty(x.shape)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(yt), nrhs), ctx)
    monkeypatch.setenv("LAGWAVE_OZ_CLUSTER", shape)
    assert L.lag_precond_dst_gemm(p, nrhs) == L.LAG_GEMM_SLICE_CLUSTER
    yc.fill_(7.0)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(yc), nrhs), ctx)
    monkeypatch.delenv("LAGWAVE_OZ_CLUSTER")
    sc = np.abs(host(yt)).max(axis=-1, keepdims=True)
    assert np.abs((host(yc) - host(yt)) / sc).max() < 1e-15
    assert np.abs((host(yt) - odst.dst_x(x)) / sc).max() < 1e-14
    assert L.lag_precond_status(p) == L.LAG_OK
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("shape", ["2x2", "1x2"])
def test_dct_f64_cluster_multicast_equals_tiles(ctx, monkeypatch, shape):
    # the cylindrical plan's forward DCT-II and its inverse (E / O sums, then the butterfly) on
    # clusters against the tile kernel (the same exact products; tail roundings grouped differently)
    nr, nz, nrhs = 300, 333, 2
    g = L.grid(nr, nz, 5.0, 4.0, cylindrical=True)
    p = C.c_void_p()
    L.check(L.lag_precond_create_sep(ctx, C.byref(g), 3e9, 3e9, 1e7, L.LAG_FP64, 0, C.byref(p)), ctx)
    x = RNG.standard_normal((nrhs, nr, nz))
    xd = dev(x)
    out = {}
    for mode in (None, shape):
        if mode:
            monkeypatch.setenv("LAGWAVE_OZ_CLUSTER", mode)
        yf, yi = empty(x.shape), empty(x.shape)
        L.check(L.lag_precond_dst(p, ptr(xd), ptr(yf), nrhs), ctx)
        L.check(L.lag_precond_dst_inverse(p, ptr(xd), ptr(yi), nrhs), ctx)
        out[mode] = (host(yf), host(yi))
        if mode:
            monkeypatch.delenv("LAGWAVE_OZ_CLUSTER")
    for a, b in zip(out[None], out[shape]):
        assert np.abs((a - b) / np.abs(a).max(axis=-1, keepdims=True)).max() < 1e-15
    assert L.lag_precond_status(p) == L.LAG_OK
    L.lag_precond_destroy(p)
