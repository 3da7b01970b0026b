"""Parity of the CUDA operator (apply_Dw / apply_Q through the C-ABI) with the oracle.

Tolerances (relative, max-norm over all compared components): 1e-10 for FP64 and
1e-5 for FP32 operator applications.
"""
import numpy as np
import pytest

from synth_inputs import WORKLOADS, GaugeConfig, kappa_to_m0, make_config, random_spinor
from oracle.dirac import WilsonDirac

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-5}


@pytest.fixture(scope="module")
def qs():
    import paper_2108_11989_gb300 as qs
    return qs


def _to_dev(psi, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(psi).view(np.float64).copy()).to(dt).cuda()


def _from_dev(t, shape):
    return t.double().cpu().numpy().view(np.complex128).reshape(shape)


def check(qs, cfg, m0, prec, nrhs, gamma5, sites=None, seed=3):
    import torch
    dt = torch.float64 if prec == "f64" else torch.float32
    lat = qs.Lattice(cfg.L, cfg.T, cfg.cstar_mask, cfg.t_antiperiodic)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    psi = random_spinor(seed, cfg.T, cfg.L, nrhs)
    if prec == "f32":
        psi = psi.astype(np.complex64).astype(np.complex128)   # the oracle sees the same inputs
    x = _to_dev(psi, dt)
    y = torch.empty_like(x)
    (lat.apply_Q if gamma5 else lat.apply_Dw)(m0, x, y)
    torch.cuda.synchronize()
    got = _from_dev(y, psi.shape).reshape(nrhs, -1, 12)
    op = WilsonDirac(cfg, lazy=sites is not None)
    fn = op.apply_Q if gamma5 else op.apply_D
    worst = 0.0
    for r in range(nrhs):
        ref = fn(psi[r].reshape(-1), m0, sites)
        ref = ref.reshape(-1, 12)
        g = got[r] if sites is None else got[r][sites]
        err = np.abs(g - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
    lat.close()
    assert worst <= TOL[prec], (prec, nrhs, gamma5, worst)
    return worst


def tiny_cfg():
    return make_config(seed=0, **WORKLOADS["tiny_4x4x4x4"])


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("gamma5", [False, True])
def test_tiny_workload(qs, prec, gamma5):
    check(qs, tiny_cfg(), kappa_to_m0(0.135), prec, 1, gamma5)


@pytest.mark.parametrize("prec,nrhs", [("f64", 3), ("f32", 5), ("f32", 4), ("f64", 2)])
def test_smallest_lattice_all_boundaries(qs, prec, nrhs):
    # 2^3 x 3: every site touches every boundary; antiperiodic t, C* in x, y only
    cfg = make_config(T=3, L=2, eps=0.8, theta_sigma=0.4, csw_su3=1.3, csw_u1=0.7, seed=9,
                      t_antiperiodic=True, cstar_mask=0b011)
    check(qs, cfg, -0.41, prec, nrhs, True)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ragged_tail(qs, prec):
    # N_s = 2 * 6^3 * 5 = 2160: not a multiple of the 128-thread block; C* in x and z
    cfg = make_config(T=5, L=6, eps=0.5, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=4,
                      cstar_mask=0b101)
    check(qs, cfg, 0.13, prec, 3, False)


def test_free_field_plane_wave_gpu(qs):
    """Closed form at a size the oracle is not needed for: free field, C* momentum."""
    import torch
    from oracle.gamma import GAMMA
    T, L = 8, 8
    su3 = np.zeros((T, L, L, L, 4, 3, 3), dtype=np.complex128)
    su3[..., 0, 0] = su3[..., 1, 1] = su3[..., 2, 2] = 1
    lat = qs.Lattice(L, T)
    lat.load_gauge(su3, None, 1.9, 0.0)
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(L), np.arange(L), np.arange(2 * L), indexing="ij")
    p1 = np.pi * 3 / L
    p = (2 * np.pi * 1 / T, p1, p1 + 2 * np.pi * 2 / L, p1 + 2 * np.pi * 5 / L)
    ph = np.exp(1j * (p[0] * t + p[1] * x + p[2] * y + p[3] * z))
    u = np.random.default_rng(0).standard_normal((4, 3)) + 0j
    psi = ph[..., None, None] * u
    m0 = -0.2
    Dp = (m0 + sum(1 - np.cos(q) for q in p)) * np.eye(4) + 1j * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
    ref = ph[..., None, None] * (Dp @ u)
    xx = _to_dev(psi, torch.float64)
    yy = torch.empty_like(xx)
    lat.apply_Dw(m0, xx, yy)
    got = _from_dev(yy, psi.shape)
    assert np.abs(got - ref).max() < 1e-12
    lat.close()


@pytest.fixture(scope="module")
def cfg16():
    return make_config(seed=0, **WORKLOADS["qcdqed_16x16x16x32"])


@pytest.mark.parametrize("prec,nrhs", [("f64", 1), ("f32", 1), ("f32", 4), ("f64", 2)])
def test_full_size_16x32_sampled(qs, cfg16, prec, nrhs):
    """16^3 x 32 (N_s = 262144) at the benchmark's launch shapes; oracle on 1500 sampled sites."""
    rng = np.random.default_rng(11)
    ns = cfg16.n_sites
    sites = np.unique(np.concatenate([rng.choice(ns, 1400, replace=False),
                                      np.arange(64), np.arange(ns - 64, ns)]))
    check(qs, cfg16, kappa_to_m0(0.135), prec, nrhs, True, sites=sites)


def test_errors(qs):
    import torch
    cfg = tiny_cfg()
    lat = qs.Lattice(cfg.L, cfg.T)
    x = torch.zeros(cfg.n_sites * 24, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(qs.QStarError) as e:     # gauge not loaded yet
        lat.apply_Dw(0.1, x, y)
    assert e.value.code == -1
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    with pytest.raises(qs.QStarError):          # in == out
        lat.apply_Dw(0.1, x, x)
    with pytest.raises(qs.QStarError):          # bad geometry: odd L
        qs.Lattice(3, 4)
    lat.close()


@pytest.mark.parametrize("prec,nrhs", [("f64", 3), ("f32", 9)])
def test_tiled_layout_matches_canonical(qs, prec, nrhs):
    """The solver's site-tiled layout gives the same operator (9 RHS: a partial group of 8)."""
    import torch
    cfg = make_config(T=4, L=4, eps=0.5, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=13)
    lat = qs.Lattice(cfg.L, cfg.T)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    dt = torch.float64 if prec == "f64" else torch.float32
    psi = random_spinor(5, cfg.T, cfg.L, nrhs)
    x = _to_dev(psi, dt).reshape(-1)
    y = torch.empty_like(x)
    lat.apply_Q(0.07, x, y)
    xt = qs.to_tiled(x, cfg.n_sites)
    yt = torch.empty_like(xt)
    lat.apply_Q(0.07, xt, yt, tiled=True)
    got = qs.from_tiled(yt, cfg.n_sites)
    assert torch.equal(got, y)
    lat.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_batched_configs_of_uneven_volume(qs, prec, tol):
    """qs_apply_Q_batch in the canonical layout (FP64: the FP64 batched kernel; FP32: the
    persistent FP32 one) = qs_apply_Q on each vector at its own mass."""
    import torch
    dt = torch.float64 if prec == "f64" else torch.float32
    cfgs = [make_config(T=4, L=4, eps=0.4, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=31),
            make_config(T=6, L=4, eps=0.3, theta_sigma=0.2, csw_su3=1.9, csw_u1=1.0, seed=32),
            make_config(T=4, L=6, eps=0.2, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=33)]
    nrhs = [2, 3, 1]
    masses = [[-0.3, 0.1], [0.05, -0.2, 0.4], [0.0]]
    lats, items, refs = [], [], []
    for cfg, nr, ms in zip(cfgs, nrhs, masses):
        lat = qs.Lattice(cfg.L, cfg.T)
        lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
        x = _to_dev(random_spinor(7 + nr, cfg.T, cfg.L, nr), dt).reshape(-1)
        y = torch.full_like(x, float("nan"))
        ref = torch.empty_like(x)
        per = cfg.n_sites * 24
        for r, m in enumerate(ms):
            lat.apply_Q(m, x[r * per:(r + 1) * per], ref[r * per:(r + 1) * per])
        lats.append(lat)
        items.append((lat, x, y, ms))
        refs.append(ref)
    qs.apply_Q_batch(items)
    torch.cuda.synchronize()
    for (_, _, y, _), ref in zip(items, refs):
        assert (y - ref).abs().max().item() <= tol * ref.abs().max().item()
    for lat in lats:
        lat.close()


# ---- 16-bit spinor storage (tiled, per-site FP32 scale), FP32 arithmetic ----------
# Tolerances (max-norm, relative to the largest output component): the output is
# rounded to 16 bits relative to its site's largest component, so the error is at most
# half a unit in the last place of the 16-bit format at 1.0 (2^-11 for FP16, 2^-8 for
# BF16) plus FP32 arithmetic; the tests allow twice that.
TOL16 = {"f16": 2 * 2.0 ** -11, "bf16": 2 * 2.0 ** -8}


def pack16(psi, kind):
    """complex [nrhs][Ns][12] -> uint8 tiles (12 x 16 words of two 16-bit reals, then 16
    FP32 scales per 16 sites) and the values the format represents (complex128)."""
    import torch
    nr, ns = psi.shape[0], psi.shape[1]
    re = np.stack([psi.real, psi.imag], axis=-1)                        # [nr][ns][12][2]
    scale = np.abs(re).reshape(nr, ns, 24).max(axis=2).astype(np.float32)
    q = re / np.where(scale > 0, scale, 1.0)[:, :, None, None]
    t = torch.from_numpy(q.astype(np.float32))
    h = t.to(torch.float16 if kind == "f16" else torch.bfloat16)
    deq = h.to(torch.float32).numpy().astype(np.float64) * scale[:, :, None, None]
    words = h.contiguous().view(torch.int16).numpy().reshape(nr, ns // 16, 16, 12, 2)
    words = words.transpose(0, 1, 3, 2, 4)                               # [nr][tile][12][16][2]
    buf = np.zeros((nr, ns // 16, 832), dtype=np.uint8)
    buf[:, :, :768] = np.ascontiguousarray(words).view(np.uint8).reshape(nr, ns // 16, 768)
    buf[:, :, 768:] = scale.reshape(nr, ns // 16, 16).view(np.uint8).reshape(nr, ns // 16, 64)
    return buf.reshape(-1), deq[..., 0] + 1j * deq[..., 1]


def unpack16(buf, nr, ns, kind):
    import torch
    b = buf.reshape(nr, ns // 16, 832)
    words = np.ascontiguousarray(b[:, :, :768]).view(np.int16).reshape(nr, ns // 16, 12, 16, 2)
    scale = np.ascontiguousarray(b[:, :, 768:]).view(np.float32).reshape(nr, ns)
    h = torch.from_numpy(np.ascontiguousarray(words.transpose(0, 1, 3, 2, 4))).view(
        torch.float16 if kind == "f16" else torch.bfloat16)
    v = h.to(torch.float32).numpy().astype(np.float64).reshape(nr, ns, 12, 2) * scale[:, :, None, None]
    return v[..., 0] + 1j * v[..., 1]


@pytest.mark.parametrize("kind", ["f16", "bf16"])
@pytest.mark.parametrize("nrhs", [1, 5])
def test_16bit_storage_against_oracle(qs, kind, nrhs):
    import torch
    # ragged volume (2160 sites = 135 tiles, not a multiple of the 128-thread block)
    cfg = make_config(T=5, L=6, eps=0.5, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=4, cstar_mask=0b101)
    lat = qs.Lattice(cfg.L, cfg.T, cfg.cstar_mask)
    lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
    ns = cfg.n_sites
    psi = random_spinor(17, cfg.T, cfg.L, nrhs).reshape(nrhs, ns, 12)
    psi[:, ::7] *= 1e-3          # sites of very different magnitude
    buf, deq = pack16(psi, kind)
    x = torch.from_numpy(buf).cuda()
    y = torch.zeros_like(x)
    prec = qs.QS_F16 if kind == "f16" else qs.QS_BF16
    m0 = -0.21
    lat.apply_Q(m0, x, y, tiled=True, prec=prec)
    got = unpack16(y.cpu().numpy(), nrhs, ns, kind)
    op = WilsonDirac(cfg)
    for r in range(nrhs):
        ref = op.apply_Q(deq[r].reshape(-1), m0).reshape(ns, 12)
        err = np.abs(got[r] - ref).max() / np.abs(ref).max()
        assert err <= TOL16[kind], (kind, r, err)
    lat.close()


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_batched_configs_against_oracle(qs, prec):
    """qs_apply_Q_batch (one persistent launch over three configurations of uneven volume,
    a mass per right-hand side) against the oracle's apply_Q at each mass."""
    import torch
    cfgs = [make_config(T=4, L=4, eps=0.4, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=31),
            make_config(T=6, L=4, eps=0.3, theta_sigma=0.2, csw_su3=1.9, csw_u1=1.0, seed=32),
            make_config(T=4, L=6, eps=0.2, theta_sigma=0.3, csw_su3=1.9, csw_u1=1.0, seed=33)]
    masses = [[-0.3, 0.1], [0.05, -0.2, 0.4], [0.0]]
    lats, items, keep = [], [], []
    for cfg, ms in zip(cfgs, masses):
        lat = qs.Lattice(cfg.L, cfg.T)
        lat.load_gauge(cfg.su3, cfg.theta, cfg.csw_su3, cfg.csw_u1)
        nr, ns = len(ms), cfg.n_sites
        psi = random_spinor(7 + nr, cfg.T, cfg.L, nr).reshape(nr, ns, 12)
        if prec == "f32":
            x = _to_dev(psi.astype(np.complex64).astype(np.complex128), torch.float32).reshape(-1)
            x = qs.to_tiled(x, ns)
            inp = psi.astype(np.complex64).astype(np.complex128)
        else:
            buf, inp = pack16(psi, "f16")
            x = torch.from_numpy(buf).cuda()
        y = torch.zeros_like(x)
        lats.append(lat)
        items.append((lat, x, y, ms))
        keep.append((cfg, inp, nr, ns))
    qs.apply_Q_batch(items, tiled=True, prec=qs.QS_F32 if prec == "f32" else qs.QS_F16)
    torch.cuda.synchronize()
    for (lat, x, y, ms), (cfg, inp, nr, ns) in zip(items, keep):
        if prec == "f32":
            got = _from_dev(qs.from_tiled(y, ns), (nr, ns, 12))
        else:
            got = unpack16(y.cpu().numpy(), nr, ns, "f16")
        op = WilsonDirac(cfg)
        for r, m in enumerate(ms):
            ref = op.apply_Q(inp[r].reshape(-1), m).reshape(ns, 12)
            err = np.abs(got[r] - ref).max() / np.abs(ref).max()
            assert err <= (TOL["f32"] if prec == "f32" else TOL16["f16"]), (prec, r, err)
    for lat in lats:
        lat.close()
