"""Mixed batch: instances of uneven size (lattice, M, K, symmetry group) in
one persistent, graph-captured launch, each instance with its own tile shape;
one p = 1 Lanczos step per instance (Sec. 3.3, Eqs. 13-17).

  - small mixed batch vs the oracle's h1, h2 and the FP64 moments / E_p1;
  - every tile shape of the engine vs the oracle;
  - equality with the single-model launches on the batch's own instances;
  - graph replay and parameter updates between replays;
  - the autotuner's choices and its invariance of the results;
  - the 64-instance mixed workload (L in {4,6,8,10}, K in {1,2},
    alpha in {1,2,4}, 256 samples each) on sampled outputs and properties.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2206_14307_gb300 import nnqs, synth
from tests.helpers import annihilated, fp32_rtol, to_complex

pytestmark = pytest.mark.gpu


def _spec(L, M, K=1, proj=False, spin_inv=0, J2=0.5, use_bias=True):
    return dict(L=L, M=M, K=K, proj_t=proj, proj_p=proj, spin_inv=spin_inv, J2=J2, use_bias=use_bias,
                precision=nnqs.FP32)


def _setup(specs, counts, seed=100, std=0.01):
    """Batch, oracle models and per-instance spins (annihilated ones replaced)."""
    b = nnqs.Batch(specs)
    oms, spins = [], []
    for i, sp in enumerate(specs):
        N = sp["L"] ** 2
        p = synth.random_params(N, sp["M"], sp["K"], std=std, seed=seed + i)
        b.models[i].set_params(p)
        oms.append(oracle.Model(sp["L"], 1.0, sp["J2"], K=sp["K"], M=sp["M"], proj_t=sp["proj_t"],
                                proj_p=sp["proj_p"], spin_inv=sp["spin_inv"], use_bias=sp["use_bias"], params=p))
        s = synth.random_sz0(N, 4 * counts[i] + 8, seed=seed + 1000 + i)
        s = s[~annihilated(sp["L"], s, sp["proj_t"], spin_inv=sp["spin_inv"], use_bias=sp["use_bias"])]
        spins.append(s[:counts[i]])
    return b, oms, spins


def _cfg(spins):
    words = [synth.pack(s) for s in spins if len(s)]
    return nnqs.cfg_tensor(np.concatenate([w.reshape(-1) for w in words])) if words else None


def _split(x, counts):
    out, o = [], 0
    for n in counts:
        out.append(x[o:o + n])
        o += n
    return out


def _check_against_oracle(oms, spins, h1, h2, rtol):
    for om, s, a1, a2 in zip(oms, spins, h1, h2):
        if not len(s):
            continue
        w1, w2 = om.lanczos_h(s)
        assert np.max(np.abs(a1 - w1) / (np.abs(w1) + 1)) <= rtol
        assert np.max(np.abs(a2 - w2) / (np.abs(w2) + 1)) <= rtol


def _assert_lanczos_close(got, moments):
    """The p = 1 step the kernel derived from its moments equals the oracle's
    closed form on the same moments: E_p1 and v to FP64 rounding, alpha to
    the cancellation of d - sqrt(d^2 + 1) at large d (near-eigenstates).
    (The moments themselves are compared separately: their central
    combinations cancel, so the step is not compared across summation
    orders.)"""
    lw = oracle.lanczos_step(np.asarray(moments[:4], np.float64))
    np.testing.assert_allclose(got[0], lw["E"], rtol=1e-12)
    np.testing.assert_allclose(got[1], lw["v"], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(got[2], lw["alpha"], rtol=1e-5, atol=1e-14)


def _moments_host(h1, h2):
    m = oracle.moments(h1, h2)["m"]
    l = oracle.lanczos_step(m)
    return m, np.array([l["E"], l["v"], l["alpha"]])


SMALL = [
    _spec(4, 16),
    _spec(4, 32, K=2, proj=True, J2=0.3),
    _spec(4, 64, proj=True, spin_inv=1, J2=0.6),
    _spec(6, 36, proj=True, J2=0.5),
    _spec(6, 72, proj=True, spin_inv=1, J2=0.1),
    _spec(4, 128, proj=True, J2=0.0, use_bias=False),
]
SMALL_COUNTS = [6, 5, 4, 2, 2, 3]


def test_small_mixed_batch_matches_oracle():
    b, oms, spins = _setup(SMALL, SMALL_COUNTS)
    cfg = _cfg(spins)
    h1, h2, mo, lz = b.lanczos(cfg, SMALL_COUNTS)
    b.status()
    H1, H2 = _split(to_complex(h1), SMALL_COUNTS), _split(to_complex(h2), SMALL_COUNTS)
    _check_against_oracle(oms, spins, H1, H2, fp32_rtol(0.01))
    mo, lz = mo.cpu().numpy(), lz.cpu().numpy()
    for i in range(len(SMALL)):
        # the batched FP64 reduction of the kernel's own h1, h2
        m, l = _moments_host(H1[i], H2[i])
        assert mo[i][4] == SMALL_COUNTS[i]
        assert abs(mo[i][7] - np.mean(np.abs(H2[i]) ** 2)) <= 1e-12 * mo[i][7]   # m4
        np.testing.assert_allclose(mo[i][:4], m[:4], rtol=1e-12, atol=1e-14)
        _assert_lanczos_close(lz[i], mo[i])
        # and the oracle's moments (E_p1 of a handful of random configurations
        # is too ill-conditioned to compare at FP32 accuracy)
        w1, w2 = oms[i].lanczos_h(spins[i])
        mw, _ = _moments_host(w1, w2)
        np.testing.assert_allclose(mo[i][1:4], mw[1:4], rtol=5e-5)


def test_mixed_batch_moments_on_sampled_configurations():
    """The batch's FP64 moments <H^n> (n = 1..4) of configurations drawn from
    |psi|^2 by the oracle's own sampler (32 per 4x4 instance, 4 per 6x6 one:
    the oracle's double enumeration of h2 is the cost) equal the oracle's
    moments of its own h1, h2 to 1e-6 relative (Sec. 3.3, Eqs. 13-17)."""
    b = nnqs.Batch(SMALL)
    counts, spins, oms = [], [], []
    for i, sp in enumerate(SMALL):
        N = sp["L"] ** 2
        p = synth.random_params(N, sp["M"], sp["K"], std=0.01, seed=900 + i)
        b.models[i].set_params(p)
        om = oracle.Model(sp["L"], 1.0, sp["J2"], K=sp["K"], M=sp["M"], proj_t=sp["proj_t"],
                          proj_p=sp["proj_p"], spin_inv=sp["spin_inv"], use_bias=sp["use_bias"], params=p)
        s, _ = om.sample(4242 + i, 4, 8, N // 2, 60) if N <= 16 else om.sample(4242 + i, 2, 2, N // 2, 60)
        oms.append(om)
        spins.append(s)
        counts.append(len(s))
    h1, h2, mo, lz = b.lanczos(_cfg(spins), counts)
    b.status()
    mo = mo.cpu().numpy()
    for i, (om, s) in enumerate(zip(oms, spins)):
        w1, w2 = om.lanczos_h(s)
        ref = oracle.moments(w1, w2)
        want = np.array([ref["m"][1], ref["m"][2], ref["m"][3], ref["m4"]])
        got = np.array([mo[i][1], mo[i][2], mo[i][3], mo[i][7]])
        assert mo[i][4] == counts[i]
        np.testing.assert_allclose(got, want, rtol=1e-6)


def _fits(v, M):
    gl, mpl = nnqs.nnqs_tile_shape(v)
    return gl * mpl


def test_every_tile_shape_matches_oracle():
    nshape = nnqs.nnqs_num_tile_shapes()
    assert nshape == 16
    widths = [_fits(v, 0) for v in range(nshape)]
    # one instance per shape, M = the shape's width (so that the shape is a candidate)
    specs = [_spec(4, widths[v], proj=(v % 2 == 0), J2=0.5, spin_inv=(v % 3 == 0) * 1) for v in range(nshape)]
    counts = [3] * nshape
    b, oms, spins = _setup(specs, counts, seed=300)
    for v in range(nshape):
        b.set_shape(v, v)
        assert b.shape(v) == v
    cfg = _cfg(spins)
    h1, h2, _, _ = b.lanczos(cfg, counts)
    b.status()
    _check_against_oracle(oms, spins, _split(to_complex(h1), counts), _split(to_complex(h2), counts),
                          fp32_rtol(0.01))


def test_shape_that_does_not_fit_is_rejected():
    b = nnqs.Batch([_spec(4, 64)])
    with pytest.raises(nnqs.NNQSError) as ei:
        b.set_shape(0, 0)  # width 16 < M
    assert ei.value.code == nnqs.NNQS_EINVAL
    with pytest.raises(nnqs.NNQSError):
        b.set_shape(0, 15)  # width 512: wider than the instance's tables
    with pytest.raises(nnqs.NNQSError):
        b.set_shape(0, 99)


def test_fp64_instance_is_unsupported():
    sp = _spec(4, 16)
    sp["precision"] = nnqs.FP64
    with pytest.raises(nnqs.NNQSError) as ei:
        nnqs.Batch([_spec(4, 16), sp])
    assert ei.value.code == nnqs.NNQS_EUNSUPPORTED


def test_batch_equals_single_model_launches():
    """Where an instance's tile shape is the single-model kernel's, the
    persistent launch does the same arithmetic in the same order as the
    single-model general engine (selected by the test hook
    NNQS_TEST_ELOC_ENGINE=old); the single-model shared-memory engine agrees
    to FP32 rounding."""
    specs = [_spec(4, 16, proj=True), _spec(6, 72, proj=True, spin_inv=1), _spec(4, 128, proj=True, K=2),
             _spec(6, 36, proj=True)]
    counts = [40, 24, 16, 0]
    b, _, spins = _setup(specs, counts, seed=500)
    cfg = _cfg(spins)
    h1, h2, mo, lz = b.lanczos(cfg, counts)
    H1, H2 = _split(to_complex(h1), counts), _split(to_complex(h2), counts)
    for i, s in enumerate(spins):
        if not len(s):
            continue
        c = nnqs.cfg_tensor(synth.pack(s))
        f1, f2, _, _ = b.models[i].lanczos(c)
        old = os.environ.get("NNQS_TEST_ELOC_ENGINE")
        os.environ["NNQS_TEST_ELOC_ENGINE"] = "old"
        try:
            g1, g2, gm, gl = b.models[i].lanczos(c)
        finally:
            if old is None:
                os.environ.pop("NNQS_TEST_ELOC_ENGINE", None)
            else:
                os.environ["NNQS_TEST_ELOC_ENGINE"] = old
        np.testing.assert_allclose(H1[i], to_complex(g1), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(H2[i], to_complex(g2), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(mo.cpu().numpy()[i][:4], gm.cpu().numpy()[:4], rtol=1e-12)
        np.testing.assert_allclose(to_complex(f1), to_complex(g1), rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(to_complex(f2), to_complex(g2), rtol=1e-5, atol=1e-5)
    # an empty instance gives m0 = 0 samples
    assert mo.cpu().numpy()[3][4] == 0


def test_graph_replay_and_parameter_update():
    b, _, spins = _setup(SMALL[:3], SMALL_COUNTS[:3], seed=700)
    counts = SMALL_COUNTS[:3]
    cfg = _cfg(spins)
    out = [torch.empty(sum(counts), 2, dtype=torch.float64, device="cuda") for _ in range(2)]
    mo = torch.empty(3, 8, dtype=torch.float64, device="cuda")
    lz = torch.empty(3, 3, dtype=torch.float64, device="cuda")
    b.lanczos(cfg, counts, out[0], out[1], mo, lz)
    first = [t.clone() for t in (out[0], out[1], mo, lz)]
    for t in (out[0], out[1], mo, lz):
        t.fill_(float("nan"))
    b.lanczos(cfg, counts, out[0], out[1], mo, lz)  # replay of the captured graph
    for a, c in zip(first, (out[0], out[1], mo, lz)):
        assert torch.equal(a, c)
    # new parameters of one instance: the replay reads the rebuilt tables
    sp = SMALL[1]
    p = synth.random_params(sp["L"] ** 2, sp["M"], sp["K"], std=0.01, seed=4242)
    b.models[1].set_params(p)
    b.lanczos(cfg, counts, out[0], out[1], mo, lz)
    om = oracle.Model(sp["L"], 1.0, sp["J2"], K=sp["K"], M=sp["M"], proj_t=True, proj_p=True, params=p)
    w1, w2 = om.lanczos_h(spins[1])
    h1 = _split(to_complex(out[0]), counts)[1]
    assert np.max(np.abs(h1 - w1) / (np.abs(w1) + 1)) <= 1e-5
    assert torch.equal(out[0][:counts[0]], first[0][:counts[0]])  # the others are unchanged


def test_autotune_picks_candidates_and_keeps_results():
    specs = [_spec(4, 64, proj=True), _spec(4, 64, proj=True, K=2), _spec(6, 72, proj=True),
             _spec(4, 100, proj=True), _spec(4, 16)]
    counts = [32, 32, 16, 16, 8]
    b, oms, spins = _setup(specs, counts, seed=900)
    cfg = _cfg(spins)
    before = [to_complex(t) for t in b.lanczos(cfg, counts)[:2]]
    shapes, ms = b.autotune(cfg, counts, probe=8)
    for i, sp in enumerate(specs):
        w = _fits(int(shapes[i]), 0)
        assert w >= sp["M"]
        assert b.shape(i) == shapes[i]
    assert shapes[0] == shapes[1]           # same size: one result shared
    assert ms[0] > 0 and ms[2] > 0 and ms[3] > 0
    assert ms[4] == 0                       # one candidate: nothing timed
    after = [to_complex(t) for t in b.lanczos(cfg, counts)[:2]]
    for x, y in zip(before, after):
        assert np.max(np.abs(x - y) / (np.abs(x) + 1)) <= 1e-5
    _check_against_oracle(oms, spins, _split(after[0], counts), _split(after[1], counts), 1e-5)


def test_mixed_workload_64_instances():
    """64 instances drawn by Philox (seed 5), 256 samples each, autotuned
    shapes, one captured launch: h1 of sampled outputs against the oracle's
    E_loc, h1/h2 of sampled outputs against the single-model launches, and
    the batched FP64 moments against the host reduction of the kernel's h1,
    h2."""
    inst = synth.mixed_batch(64, seed=5)
    specs = [_spec(d["L"], d["M"], K=d["K"], proj=True, J2=d["J2"]) for d in inst]
    counts = [256] * 64
    b = nnqs.Batch(specs)
    spins = []
    for i, (d, sp) in enumerate(zip(inst, specs)):
        N = d["L"] ** 2
        b.models[i].set_params(synth.random_params(N, d["M"], d["K"], std=0.01, seed=5000 + i))
        c, _ = b.models[i].sample(14307 + i, 16, 16, 10, 100)
        spins.append(synth.unpack(c.cpu().numpy().view(np.uint64), N))
    cfg = _cfg(spins)
    shapes, ms = b.autotune(cfg, counts, probe=64)
    h1, h2, mo, lz = b.lanczos(cfg, counts)
    b.status()
    H1, H2 = _split(to_complex(h1), counts), _split(to_complex(h2), counts)
    mo, lz = mo.cpu().numpy(), lz.cpu().numpy()
    rng = np.random.default_rng(55)
    for i, d in enumerate(inst):
        m, l = _moments_host(H1[i], H2[i])
        np.testing.assert_allclose(mo[i][:4], m[:4], rtol=1e-12, atol=1e-14)
        _assert_lanczos_close(lz[i], mo[i])
        assert mo[i][4] == 256
        assert np.all(np.isfinite(H1[i])) and np.all(np.isfinite(H2[i]))
    # sampled outputs against the single-model launches (h1 and h2)
    for i in rng.choice(64, 8, replace=False):
        k = rng.choice(256, 2, replace=False)
        c = nnqs.cfg_tensor(synth.pack(spins[i][k]))
        g1, g2, _, _ = b.models[i].lanczos(c)
        assert np.max(np.abs(H1[i][k] - to_complex(g1)) / (np.abs(to_complex(g1)) + 1)) <= 1e-5
        assert np.max(np.abs(H2[i][k] - to_complex(g2)) / (np.abs(to_complex(g2)) + 1)) <= 1e-5
    # h1 = E_loc of one sample of one instance per lattice size against the oracle
    for L in (4, 6, 8, 10):
        i = next(j for j, d in enumerate(inst) if d["L"] == L)
        d = inst[i]
        om = oracle.Model(L, 1.0, d["J2"], K=d["K"], M=d["M"], proj_t=True, proj_p=True,
                          params=synth.random_params(L * L, d["M"], d["K"], std=0.01, seed=5000 + i))
        want = om.local_energy(spins[i][:1])
        assert np.max(np.abs(H1[i][:1] - want) / (np.abs(want) + 1)) <= 1e-5
