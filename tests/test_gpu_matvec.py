"""GPU parity of K u against the FP64 oracle (through the C ABI).

Tolerances: relative L2 <= 1e-12 for FP64, <= 2e-5 for FP32 (the inputs are
rounded to FP32 first, so the FP32 check measures the kernel's own error).
Sizes span several CTA tiles and leave ragged tails in every direction.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn
from helpers import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pd():
    import paper_2301_11828_gb300 as pd
    pd.load_library()
    assert torch.cuda.is_available()
    return pd


TOL = {torch.float64: 1e-12, torch.float32: 2e-5}


def _oracle_K(dim, n, h, M, u, cons=None, E=None, mu=None, Efield=None):
    if Efield is not None:
        al1 = oracle.alpha(dim, 1.0, M * h)
        return oracle.stiffness(dim, n, h, M, al1, u, cons=cons, E=Efield, mu=mu)
    al = oracle.alpha(dim, E if E is not None else 1.0, M * h)
    return oracle.stiffness(dim, n, h, M, al, u, cons=cons, mu=mu)


def _run(pd, g, u_np, dtype, flags):
    u = torch.tensor(u_np, dtype=dtype, device="cuda")
    out = g.matvec(u, flags=flags)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), u.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,M", [((67, 45), 1), ((67, 45), 2), ((130, 97), 3), ((129, 70), 4), ((75, 66), 5),
                                 ((80, 91), 6), ((70, 70), 7), ((99, 53), 8), ((5, 3), 3), ((1, 1), 2),
                                 ((1, 40), 3), ((200, 2), 4)])
def test_stencil_2d_matches_oracle(pd, dtype, n, M):
    h = 1.0 / 64
    rng = np.random.default_rng(M * 1000 + n[0])
    u_np = rng.uniform(-1, 1, (2, n[1], n[0]))
    g = pd.Grid(2, n, h, M, E=2.5)
    out, u_used = _run(pd, g, u_np, dtype, pd.PD_METHOD_STENCIL)
    ref = _oracle_K(2, n, h, M, u_used, E=2.5)
    assert rel_l2(out, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_stencil_2d_projection(pd, dtype):
    w = syn.plate_static(97, 3, tag=5, u_amp=1.0)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    out, u_used = _run(pd, g, w.u, dtype, pd.PD_METHOD_STENCIL | pd.PD_PROJECT)
    ref = _oracle_K(2, w.n, w.h, w.M, u_used, cons=w.constrained)
    assert rel_l2(out, ref) <= TOL[dtype]
    assert np.all(out[w.constrained.astype(bool)] == 0)
    # without the flag the constraint is not applied
    out2, _ = _run(pd, g, w.u, dtype, pd.PD_METHOD_STENCIL)
    assert rel_l2(out2, _oracle_K(2, w.n, w.h, w.M, u_used)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,M", [((37, 19, 13), 1), ((37, 19, 13), 2), ((40, 21, 19), 3), ((35, 17, 22), 4),
                                 ((3, 2, 5), 3), ((1, 1, 1), 1)])
def test_stencil_3d_matches_oracle(pd, dtype, n, M):
    h = 1.0 / 32
    rng = np.random.default_rng(M + 7 * n[0])
    u_np = rng.uniform(-1, 1, (3, n[2], n[1], n[0]))
    g = pd.Grid(3, n, h, M)
    out, u_used = _run(pd, g, u_np, dtype, pd.PD_METHOD_STENCIL)
    ref = _oracle_K(3, n, h, M, u_used)
    assert rel_l2(out, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_stencil_3d_projection(pd, dtype):
    w = syn.cube(24, 3)
    g = pd.Grid(3, w.n, w.h, w.M, constrained=w.constrained)
    out, u_used = _run(pd, g, w.u, dtype, pd.PD_METHOD_STENCIL | pd.PD_PROJECT)
    ref = _oracle_K(3, w.n, w.h, w.M, u_used, cons=w.constrained)
    assert rel_l2(out, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("M", [3, 4])
def test_modulus_field_direct_form(pd, dtype, M):
    """Per-node modulus: bond (p,q) uses (E_p + E_q)/2 (the direct kernel)."""
    n = (83, 71)
    h = 1.0 / 80
    E = syn.lognormal_modulus(n, 0.1, 31)
    rng = np.random.default_rng(3)
    u_np = rng.uniform(-1, 1, (2, n[1], n[0]))
    g = pd.Grid(2, n, h, M, E_field=torch.tensor(E, device="cuda"))
    out, u_used = _run(pd, g, u_np, dtype, 0)
    ref = _oracle_K(2, n, h, M, u_used, Efield=E)
    assert rel_l2(out, ref) <= TOL[dtype]


def _random_broken_state(pd, g, n, h, M, dim, seed, sigma=0.05):
    """Break a scattered set of bonds with the library, return the oracle mu."""
    rng = np.random.default_rng(seed)
    u_np = rng.normal(0, sigma * h, (dim,) + tuple(reversed(n)))
    g.set_material(E=1.0, s0=0.03)
    nb = g.break_bonds(torch.tensor(u_np, device="cuda"))
    mu = oracle.intact_mu(dim, n, M)
    nb_or = oracle.break_bonds(dim, n, h, M, 0.03, u_np, mu)
    assert nb == nb_or and nb > 0
    return mu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("dim,n,M", [(2, (90, 77), 3), (2, (70, 66), 5), (3, (30, 21, 17), 2)])
def test_broken_bonds_df_gather(pd, dtype, dim, n, M):
    """TBT stencil + sparse D^f gather equals the oracle's bond sum with mu."""
    h = 1.0 / 64
    g = pd.Grid(dim, n, h, M)
    mu = _random_broken_state(pd, g, n, h, M, dim, seed=11 + M)
    rng = np.random.default_rng(5)
    u_np = rng.uniform(-1, 1, (dim,) + tuple(reversed(n)))
    out, u_used = _run(pd, g, u_np, dtype, pd.PD_METHOD_STENCIL)
    ref = _oracle_K(dim, n, h, M, u_used, mu=mu)
    assert rel_l2(out, ref) <= TOL[dtype]
    # ignoring the broken bonds gives the intact operator
    out0, _ = _run(pd, g, u_np, dtype, pd.PD_METHOD_STENCIL | pd.PD_IGNORE_BROKEN)
    assert rel_l2(out0, _oracle_K(dim, n, h, M, u_used)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_broken_bonds_with_modulus_field(pd, dtype):
    n, M, h = (77, 64), 3, 1.0 / 64
    E = syn.lognormal_modulus(n, 0.1, 8)
    g = pd.Grid(2, n, h, M, E_field=torch.tensor(E, device="cuda"))
    rng = np.random.default_rng(4)
    u_b = rng.normal(0, 0.05 * h, (2, n[1], n[0]))
    g.set_material(E=1.0, s0=0.03, E_field=torch.tensor(E, device="cuda"))
    g.break_bonds(torch.tensor(u_b, device="cuda"))
    mu = oracle.intact_mu(2, n, M)
    oracle.break_bonds(2, n, h, M, 0.03, u_b, mu)
    u_np = rng.uniform(-1, 1, (2, n[1], n[0]))
    out, u_used = _run(pd, g, u_np, dtype, 0)
    ref = _oracle_K(2, n, h, M, u_used, mu=mu, Efield=E)
    assert rel_l2(out, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_matvec_equals_single(pd, dtype):
    n, M, h = (70, 45), 3, 1.0 / 64
    g = pd.Grid(2, n, h, M)
    rng = np.random.default_rng(9)
    U = torch.tensor(rng.uniform(-1, 1, (5, 2, n[1], n[0])), dtype=dtype, device="cuda")
    out = g.matvec(U, flags=pd.PD_METHOD_STENCIL)
    for b in range(5):
        single = g.matvec(U[b].contiguous(), flags=pd.PD_METHOD_STENCIL)
        assert torch.equal(out[b], single)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("M", [3, 6])
def test_full_size_plate_1024(pd, dtype, M):
    """The 1024 x 1024 plate at delta = 3h and 6h, whole field against the oracle."""
    w = syn.large_plate(M)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    out, u_used = _run(pd, g, w.u, dtype, pd.PD_METHOD_STENCIL | pd.PD_PROJECT)
    ref = _oracle_K(2, w.n, w.h, w.M, u_used, cons=w.constrained)
    assert rel_l2(out, ref) <= TOL[dtype]


def test_full_size_cube_128_sampled(pd):
    """128^3 cube, FP32: whole-field relative error, and FP64 on a sampled slab."""
    w = syn.cube(128, 3)
    g = pd.Grid(3, w.n, w.h, w.M, constrained=w.constrained)
    out, u_used = _run(pd, g, w.u, torch.float32, pd.PD_METHOD_STENCIL | pd.PD_PROJECT)
    ref = _oracle_K(3, w.n, w.h, w.M, u_used, cons=w.constrained)
    assert rel_l2(out, ref) <= 2e-5
    out64, u64 = _run(pd, g, w.u, torch.float64, pd.PD_METHOD_STENCIL | pd.PD_PROJECT)
    ref64 = _oracle_K(3, w.n, w.h, w.M, u64, cons=w.constrained)
    assert rel_l2(out64, ref64) <= 1e-12


# ----------------------------------------------------------------------------- bond state (bit-exact)

@pytest.mark.parametrize("dim,n,M,dtype", [(2, (150, 131), 3, torch.float64), (2, (64, 70), 6, torch.float64),
                                           (2, (90, 80), 4, torch.float32), (3, (33, 20, 18), 3, torch.float64)])
def test_break_bonds_bit_exact(pd, dim, n, M, dtype):
    """Broken sets equal the oracle's bit for bit (same FP64 operation order)."""
    from helpers import mask_to_mu
    h = 1.0 / 128
    rng = np.random.default_rng(21)
    g = pd.Grid(dim, n, h, M, s0=1e-3)
    mu = oracle.intact_mu(dim, n, M)
    total = 0
    for it in range(3):
        u_np = rng.normal(0, 1.5e-3 * h, (dim,) + tuple(reversed(n)))
        u_t = torch.tensor(u_np, dtype=dtype, device="cuda")
        u_used = u_t.double().cpu().numpy()
        nb = g.break_bonds(u_t)
        nb_or = oracle.break_bonds(dim, n, h, M, 1e-3, u_used, mu)
        assert nb == nb_or
        total += nb
        got = mask_to_mu(g.bond_mask().cpu().numpy(), g.nnb)
        assert np.array_equal(got, mu)
    assert total > 0
    assert np.array_equal(g.offsets(), oracle.offsets(dim, M))


@pytest.mark.parametrize("dim,n,M", [(2, (48, 40), 3), (2, (33, 29), 5), (3, (14, 12, 10), 3)])
def test_break_near_threshold_bit_exact(pd, dim, n, M):
    """Stretches within a few ulps of s0: the kernel's per-offset threshold on
    |xi + eta|^2 must decide exactly as the oracle's square root and division do.
    A uniform stretch by (1 + s0) puts every bond on the threshold; perturbations of
    1e-16 .. 1e-13 (relative) scatter them to both sides."""
    from helpers import mask_to_mu
    h = 1.0 / 64
    s0 = 1e-3
    rng = np.random.default_rng(77)
    for trial, rel in enumerate((1e-16, 1e-15, 1e-14, 1e-13)):
        g = pd.Grid(dim, n, h, M, s0=s0)
        mu = oracle.intact_mu(dim, n, M)
        coords = np.meshgrid(*[(np.arange(k) + 0.5) * h for k in reversed(n)], indexing="ij")[::-1]
        u_np = np.stack([s0 * c for c in coords]) * (1 + rel * rng.standard_normal((dim,) + tuple(reversed(n))))
        u_t = torch.tensor(u_np, dtype=torch.float64, device="cuda")
        nb = g.break_bonds(u_t)
        nb_or = oracle.break_bonds(dim, n, h, M, s0, u_np, mu)
        assert nb == nb_or
        got = mask_to_mu(g.bond_mask().cpu().numpy(), g.nnb)
        assert np.array_equal(got, mu)
        n_pairs = mu.size // 2
        assert 0 < nb_or < n_pairs, (rel, nb_or)   # both sides of the threshold occur


@pytest.mark.parametrize("nside", [32, 512])
def test_prenotch_bit_exact(pd, nside):
    from helpers import mask_to_mu
    w = syn.crack_plate(nside, 3)
    g = pd.Grid(2, w.n, w.h, w.M)
    nb = g.break_segment(w.extra["notch"], w.extra["notch_den"])
    mu = oracle.intact_mu(2, w.n, w.M)
    nb_or = oracle.prenotch(w.n, w.M, w.extra["notch"], w.extra["notch_den"], mu)
    assert nb == nb_or
    assert np.array_equal(mask_to_mu(g.bond_mask().cpu().numpy(), g.nnb), mu)


def test_bond_mask_roundtrip(pd):
    from helpers import mu_to_mask
    n, M, h = (40, 33), 3, 1.0 / 32
    g = pd.Grid(2, n, h, M)
    rng = np.random.default_rng(2)
    mu = oracle.intact_mu(2, n, M)
    oracle.break_bonds(2, n, h, M, 0.02, rng.normal(0, 0.02 * h, (2, n[1], n[0])), mu)
    g.set_bond_mask(torch.tensor(mu_to_mask(mu), device="cuda"))
    u_np = rng.uniform(-1, 1, (2, n[1], n[0]))
    out, u_used = _run(pd, g, u_np, torch.float64, pd.PD_METHOD_STENCIL)
    assert rel_l2(out, _oracle_K(2, n, h, M, u_used, mu=mu)) <= 1e-12


@pytest.mark.parametrize("n,M", [((64, 64), 1), ((128, 36), 2), ((200, 2), 3), ((4, 1), 3), ((68, 131), 4),
                                 ((256, 96), 5), ((96, 70), 6), ((132, 67), 7), ((100, 100), 8)])
def test_tma_stencil_matches_plain_and_oracle(pd, n, M):
    """FP32 rows that are a multiple of 4 floats take the TMA-fed kernel; it agrees
    with the plain kernel and with the oracle, with projection and a batch."""
    h = 1.0 / 64
    rng = np.random.default_rng(M + n[0])
    cons = (rng.random((2, n[1], n[0])) < 0.1).astype(np.uint8)
    g = pd.Grid(2, n, h, M, constrained=cons)
    U = torch.tensor(rng.uniform(-1, 1, (3, 2, n[1], n[0])), dtype=torch.float32, device="cuda")
    for proj in (0, pd.PD_PROJECT):
        plain = g.matvec(U, flags=pd.PD_METHOD_STENCIL | proj | pd.PD_NO_TMA)
        for form in (0, pd.PD_PAIR_FORM):   # the default difference form and the pair form of the TMA kernel
            fast = g.matvec(U, flags=pd.PD_METHOD_STENCIL | proj | form)
            torch.cuda.synchronize()
            assert rel_l2(fast.double().cpu().numpy(), plain.double().cpu().numpy()) <= 2e-6
            for b in range(3):
                ub = U[b].double().cpu().numpy()
                ref = _oracle_K(2, n, h, M, ub, cons=cons if proj else None)
                assert rel_l2(fast[b].double().cpu().numpy(), ref) <= 2e-5


@pytest.mark.parametrize("M", [2, 3])
def test_accurate_form_3d(pd, M):
    """The 3D stencil's difference form: parity on random fields (with projection),
    and a much smaller interior error than the pair form on a smooth field."""
    n, h = (40, 33, 29), 1.0 / 64
    rng = np.random.default_rng(M)
    w = syn.cube(24, M)
    cons = (rng.random((3, n[2], n[1], n[0])) < 0.05).astype(np.uint8)
    g = pd.Grid(3, n, h, M, constrained=cons)
    ut = torch.tensor(rng.uniform(-1, 1, (3, n[2], n[1], n[0])), dtype=torch.float32, device="cuda")
    for proj in (0, pd.PD_PROJECT):
        out = g.matvec(ut, flags=pd.PD_METHOD_STENCIL | pd.PD_ACCURATE | proj).double().cpu().numpy()
        ref = _oracle_K(3, n, h, M, ut.double().cpu().numpy(), cons=cons if proj else None)
        assert rel_l2(out, ref) <= 2e-5
    x = (np.arange(n[0]) + 0.5) / n[0]
    y = (np.arange(n[1]) + 0.5) / n[1]
    z = (np.arange(n[2]) + 0.5) / n[2]
    sm = np.sin(2 * np.pi * x)[None, None, :] * np.cos(np.pi * y)[None, :, None] * np.cos(np.pi * z)[:, None, None]
    us = torch.tensor(np.stack([sm, 0.5 * sm, -sm]), dtype=torch.float32, device="cuda")
    ref = _oracle_K(3, n, h, M, us.double().cpu().numpy())
    acc = g.matvec(us, flags=pd.PD_METHOD_STENCIL).double().cpu().numpy()
    pair = g.matvec(us, flags=pd.PD_METHOD_STENCIL | pd.PD_PAIR_FORM).double().cpu().numpy()
    inner = (slice(None), slice(M, -M), slice(M, -M), slice(M, -M))
    assert rel_l2(acc[inner], ref[inner]) * 10 <= rel_l2(pair[inner], ref[inner])
    assert rel_l2(acc, ref) <= 2e-5


def _smooth_field(n, offset):
    """A smooth displacement field: one to one-and-a-half waves across the
    plate per component, optionally on top of a large constant part (a rigid
    translation, which K maps to zero)."""
    x = (np.arange(n[0]) + 0.5) / n[0]
    y = (np.arange(n[1]) + 0.5) / n[1]
    a = np.sin(2 * np.pi * x)[None, :] * np.cos(np.pi * y)[:, None]
    b = np.cos(3 * np.pi * x)[None, :] * np.sin(2 * np.pi * y)[:, None]
    if offset:
        return np.stack([1.0 + 0.3 * a, 0.7 + 0.2 * b])
    return np.stack([a, b])


@pytest.mark.parametrize("n", [(512, 384), (1024, 1024)])
@pytest.mark.parametrize("M", [3, 6])
@pytest.mark.parametrize("offset", [False, True])
def test_accurate_form_on_smooth_fields(pd, n, M, offset):
    """The default FP32 product (the kernel the benchmark times) sums differences
    of nearby values, so its FP32 error stays relative to |K u| on smooth fields
    and on fields with a large constant part, where the terms of the pair form
    Kd u_p - sum c (u_p+o + u_p-o) cancel.  Whole field and full-horizon
    interior, against the FP64 oracle on the same FP32 input; the pair form
    (PD_PAIR_FORM, kept for comparison) misses the tolerance here."""
    h = 1.0 / n[0]
    g = pd.Grid(2, n, h, M)
    ut = torch.tensor(_smooth_field(n, offset), dtype=torch.float32, device="cuda")
    ref = _oracle_K(2, n, h, M, ut.double().cpu().numpy())
    acc = g.matvec(ut, flags=pd.PD_METHOD_STENCIL).double().cpu().numpy()
    pair = g.matvec(ut, flags=pd.PD_METHOD_STENCIL | pd.PD_PAIR_FORM).double().cpu().numpy()
    inner = (slice(None), slice(M, n[1] - M), slice(M, n[0] - M))
    e_acc, e_acc_in = rel_l2(acc, ref), rel_l2(acc[inner], ref[inner])
    e_pair_in = rel_l2(pair[inner], ref[inner])
    print(f"n={n} M={M} offset={offset}: default {e_acc:.3e} (interior {e_acc_in:.3e}), "
          f"pair form interior {e_pair_in:.3e}")
    assert e_acc <= 2e-5 and e_acc_in <= 2e-5
    assert e_acc <= 1e-6 and e_acc_in <= 1e-6      # in fact about 1e-7
    assert e_pair_in > 2e-5


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batch_from_host_memory(pd, dtype):
    """pd_matvec_batch_host (chunks uploaded, multiplied and downloaded on three
    streams) gives the same bits as the device call, pinned or pageable, for
    batches that do and do not divide into chunks."""
    w = syn.plate_static(256, 3, tag=2, u_amp=1.0)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    fl = (pd.PD_F32 if dtype == torch.float32 else pd.PD_F64) | pd.PD_PROJECT
    rng = np.random.default_rng(12)
    for B, pin in ((1, True), (7, True), (33, False)):
        U = torch.tensor(rng.uniform(-1, 1, (B, 2, w.n[1], w.n[0])), dtype=dtype)
        if pin:
            U = U.pin_memory()
        O = torch.empty_like(U)
        if pin:
            O = O.pin_memory()
        pd.pd_matvec_batch_host(g.handle, B, U, O, fl)
        torch.cuda.synchronize()
        Ud = U.cuda()
        Od = torch.empty_like(Ud)
        pd.pd_matvec_batch(g.handle, B, Ud, Od, fl)
        torch.cuda.synchronize()
        assert torch.equal(O, Od.cpu())


def test_headline_launch_configuration_sampled(pd):
    """The timed configuration itself: 32 fields of the 1024^2 plate (delta = 3h,
    FP32, TMA stencil) in one batched launch; three of the fields (first, middle,
    last) are checked in full against the oracle."""
    w = syn.large_plate(3)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    B = 32
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    U = torch.empty((B, 2, w.n[1], w.n[0]), dtype=torch.float32, device="cuda")
    U.uniform_(-1.0, 1.0, generator=gen)
    O = torch.empty_like(U)
    pd.pd_matvec_batch(g.handle, B, U, O, pd.PD_F32 | pd.PD_METHOD_STENCIL)
    torch.cuda.synchronize()
    al = oracle.alpha(2, 1.0, w.delta)
    for b in (0, 17, 31):
        ref = oracle.stiffness(2, w.n, w.h, w.M, al, U[b].double().cpu().numpy())
        assert rel_l2(O[b].double().cpu().numpy(), ref) <= 2e-5


def test_headline_launch_configuration_smooth_fields(pd):
    """The timed configuration (32 fields of the 1024^2 plate in one batched
    launch, default FP32 product) on smooth fields with and without a constant
    part: every field within the FP32 tolerance of the oracle, whole field."""
    w = syn.large_plate(3)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    B = 32
    fields = [_smooth_field(w.n, False), _smooth_field(w.n, True)]
    U = torch.empty((B, 2, w.n[1], w.n[0]), dtype=torch.float32, device="cuda")
    for b in range(B):
        U[b] = torch.tensor(fields[b % 2] * (1.0 + 0.01 * b), dtype=torch.float32)
    O = torch.empty_like(U)
    pd.pd_matvec_batch(g.handle, B, U, O, pd.PD_F32 | pd.PD_METHOD_STENCIL)
    torch.cuda.synchronize()
    al = oracle.alpha(2, 1.0, w.delta)
    for b in (0, 1, 30, 31):
        ref = oracle.stiffness(2, w.n, w.h, w.M, al, U[b].double().cpu().numpy())
        assert rel_l2(O[b].double().cpu().numpy(), ref) <= 2e-5


@pytest.mark.parametrize("t", [0.4, 2.5])
def test_plate_thickness_parity(pd, t):
    """A plate of thickness t != 1: alpha carries 1/t and the node volume h^2 t
    (Sec. 2.1, Eq. mat:f1); the product matches the oracle built from the same
    two factors, in FP64 and FP32, by stencil and FFT."""
    n, M, E = (70, 52), 3, 1.7
    h = 1.0 / 64
    rng = np.random.default_rng(int(10 * t))
    u = rng.uniform(-1, 1, (2, n[1], n[0]))
    g = pd.Grid(2, n, h, M, E=E, thickness=t)
    ref = oracle.stiffness(2, n, h, M, oracle.bond_constant(2, E, M * h, t), u)
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
        ut = torch.tensor(u, dtype=dt, device="cuda")
        r = oracle.stiffness(2, n, h, M, oracle.bond_constant(2, E, M * h, t), ut.double().cpu().numpy())
        for meth in (pd.PD_METHOD_STENCIL, pd.PD_METHOD_FFT):
            out = g.matvec(ut, flags=meth).double().cpu().numpy()
            assert rel_l2(out, r) <= tol
    assert rel_l2(ref, oracle.stiffness(2, n, h, M, oracle.alpha(2, E, M * h), u)) < 1e-14


@pytest.mark.parametrize("offset", [False, True])
def test_3d_products_on_smooth_fields(pd, offset):
    """3D: the default FP32 stencil (difference form, out-of-grid terms dropped)
    and the FP32 FFT tiles (16^3 tiles of u - c: 4e-6 here, 1e-5 on the 128^3 cube;
    their error grows like 1/h, so the autotuner does not pick them in FP32)
    within the FP32 tolerance on a smooth field with and without a constant
    part; the FP64 stencil and FFT tiles within the FP64 tolerance."""
    n, M = (64, 48, 40), 3
    h = 1.0 / 64
    x = (np.arange(n[0]) + 0.5) / n[0]
    y = (np.arange(n[1]) + 0.5) / n[1]
    z = (np.arange(n[2]) + 0.5) / n[2]
    sm = np.sin(2 * np.pi * x)[None, None, :] * np.cos(np.pi * y)[None, :, None] * np.cos(np.pi * z)[:, None, None]
    u = np.stack([sm, 0.5 * sm, -sm])
    if offset:
        u = 0.3 * u + np.array([1.0, 0.7, -0.5])[:, None, None, None]
    g = pd.Grid(3, n, h, M)
    for dt, tol, meths in ((torch.float32, 2e-5, (pd.PD_METHOD_STENCIL, pd.PD_METHOD_FFT)),
                           (torch.float64, 1e-12, (pd.PD_METHOD_STENCIL, pd.PD_METHOD_FFT))):
        ut = torch.tensor(u, dtype=dt, device="cuda")
        ref = _oracle_K(3, n, h, M, ut.double().cpu().numpy())
        for meth in meths:
            out = g.matvec(ut, flags=meth).double().cpu().numpy()
            assert rel_l2(out, ref) <= tol, (str(dt), meth)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,M", [((130, 97), 3), ((75, 66), 5), ((99, 53), 8)])
def test_pair_form_plain_kernel(pd, dtype, n, M):
    """PD_PAIR_FORM on the plain 2D kernel (FP64, and FP32 off the TMA path):
    Kd_p u_p - sum c (u_p+o + u_p-o) with the clipped-distance diagonal, against
    the oracle on random fields, with and without projection (the FP64 CG and
    ADR iterations use this form)."""
    h = 1.0 / 64
    rng = np.random.default_rng(7 * M + n[0])
    u_np = rng.uniform(-1, 1, (2, n[1], n[0]))
    cons = syn.clamp_left(2, n, M)
    g = pd.Grid(2, n, h, M, constrained=cons)
    for proj in (0, pd.PD_PROJECT):
        out, u_used = _run(pd, g, u_np, dtype, pd.PD_METHOD_STENCIL | pd.PD_PAIR_FORM | pd.PD_NO_TMA | proj)
        ref = _oracle_K(2, n, h, M, u_used, cons=cons if proj else None)
        assert rel_l2(out, ref) <= TOL[dtype]


def _linear_part(n, gx, gy, c0):
    x = np.arange(n[0], dtype=np.float64)[None, :]
    y = np.arange(n[1], dtype=np.float64)[:, None]
    return c0 + gx * x / n[0] + gy * y / n[1]


@pytest.mark.parametrize("n,M", [((512, 384), 3), ((1024, 1024), 3), ((300, 217), 6), ((130, 97), 2.5)])
@pytest.mark.parametrize("kind", ["smooth", "offset", "gradient"])
def test_f64_plane_pair_form_on_smooth_fields(pd, n, M, kind):
    """The default FP64 2D product is the pair form on u minus each box's
    least-squares plane (exact in FP64), with K of the plane added at the nodes
    near a face from the first-moment table: within 1e-12 of the oracle on
    smooth fields, on fields with a large constant part and on fields with a
    large linear part (where K of the plane at the faces is large), whole field
    and full-horizon interior, with and without projection.  The difference
    form (PD_ACCURATE) and the pair form on u itself (PD_PAIR_FORM) are printed
    beside it (the latter reaches 3e-10 on the interior of the linear case)."""
    h = 1.0 / n[0]
    u_np = _smooth_field(n, kind != "smooth")
    if kind == "gradient":
        u_np = u_np + np.stack([_linear_part(n, 40.0, -25.0, 5.0), _linear_part(n, -30.0, 60.0, -3.0)])
    cons = syn.clamp_left(2, n, int(np.ceil(M)))
    g = pd.Grid(2, n, h, M, constrained=cons)
    Mi = g.M
    ut = torch.tensor(u_np, dtype=torch.float64, device="cuda")
    inner = (slice(None), slice(Mi, n[1] - Mi), slice(Mi, n[0] - Mi))
    for proj in (0, pd.PD_PROJECT):
        ref = _oracle_K(2, n, h, M, u_np, cons=cons if proj else None)
        res = {}
        for name, fl in (("default", 0), ("difference", pd.PD_ACCURATE), ("pair", pd.PD_PAIR_FORM)):
            out = g.matvec(ut, flags=pd.PD_METHOD_STENCIL | proj | fl).cpu().numpy()
            res[name] = (rel_l2(out, ref), rel_l2(out[inner], ref[inner]))
        print(f"n={n} M={M} {kind} proj={bool(proj)}: " +
              ", ".join(f"{k} {v[0]:.2e} (interior {v[1]:.2e})" for k, v in res.items()))
        e, e_in = res["default"]
        assert e <= 1e-12 and e_in <= 1e-12
        assert res["difference"][0] <= 1e-12


@pytest.mark.parametrize("n,M", [((131, 70), 3), ((64, 33), 4), ((3, 70), 2), ((70, 3), 8)])
def test_f64_plane_pair_form_matches_difference_form(pd, n, M):
    """Random fields: the plane-subtracted pair form and the difference form
    agree to FP64 rounding, in a batch and alone."""
    rng = np.random.default_rng(3 * M + n[0])
    U = torch.tensor(rng.uniform(-1, 1, (3, 2, n[1], n[0])), dtype=torch.float64, device="cuda")
    g = pd.Grid(2, n, 1.0 / 64, M)
    a = g.matvec(U, flags=pd.PD_METHOD_STENCIL)
    d = g.matvec(U, flags=pd.PD_METHOD_STENCIL | pd.PD_ACCURATE)
    one = g.matvec(U[1].contiguous(), flags=pd.PD_METHOD_STENCIL)
    torch.cuda.synchronize()
    assert torch.equal(one, a[1])
    assert rel_l2(a.cpu().numpy(), d.cpu().numpy()) <= 1e-14
    ref = _oracle_K(2, n, 1.0 / 64, M, U[2].cpu().numpy())
    assert rel_l2(a[2].cpu().numpy(), ref) <= 1e-13


@pytest.mark.parametrize("method", ["stencil", "fft"])
def test_modulus_change_rebuilds_plane_tables(pd, method):
    """The first-moment tables that give K of a tile's plane at the faces
    (FP64 stencil, FP32 FFT tiles) scale with the modulus: after
    pd_set_material changes E, products of a field with a large gradient
    still match the oracle at the new modulus."""
    n, h = (200, 150), 1.0 / 200
    M = 3 if method == "stencil" else 6   # the FP32 FFT tiles serve the larger horizons
    g = pd.Grid(2, n, h, M)
    u_np = _smooth_field(n, True) + np.stack([_linear_part(n, 40.0, -25.0, 5.0), _linear_part(n, -30.0, 60.0, -3.0)])
    meth = pd.PD_METHOD_STENCIL if method == "stencil" else pd.PD_METHOD_FFT
    dt = torch.float64 if method == "stencil" else torch.float32
    tol = 1e-12 if method == "stencil" else 2e-5
    for E in (1.0, 3.5):
        g.set_material(E=E)
        ut = torch.tensor(u_np, dtype=dt, device="cuda")
        out = g.matvec(ut, flags=meth).double().cpu().numpy()
        ref = _oracle_K(2, n, h, M, ut.double().cpu().numpy(), E=E)
        assert rel_l2(out, ref) <= tol, (E, rel_l2(out, ref))
