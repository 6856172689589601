"""Batched updates with ragged grids and history lengths in one persistent
convolution launch (and a captured CUDA graph), through the C ABI: bit-equal
to the members stepped one by one with the same lag chunking, and within the
FP32 bound of the oracle."""
import numpy as np
import pytest

from oracle.sbim_oracle import SBIMOracle
from paper_2102_08756_gb300.synth import separable_history
from tests._errors import assert_finite

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CS, CP, RHO = 3464.0, 6000.0, 2670.0
MEMBERS = [(16, 16, 5, 1), (32, 24, 17, -1), (8, 8, 40, 1), (24, 24, 3, -1), (16, 32, 64, 1)]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _setup(stream, precision=1, kahan=1):
    from paper_2102_08756_gb300 import sbim as B
    dx = 100.0
    dt = 0.3 * dx / CP
    n1 = [m[0] for m in MEMBERS]
    n3 = [m[1] for m in MEMBERS]
    b = B.sbim_batch_create(n1, n3, [x * dx for x in n1], [x * dx for x in n3], [CS] * 5, [CP] * 5,
                            [RHO] * 5, [dt] * 5, [m[2] for m in MEMBERS], [m[3] for m in MEMBERS],
                            precision, kahan, stream.cuda_stream)
    hist = [separable_history(a, c, a * dx, c * dx, 80, dt, CS, seed=10 + k, spectrum="k2")
            for k, (a, c, _, _) in enumerate(MEMBERS)]
    return B, b, hist, dt


def _fields(hist, m):
    u = [torch.from_numpy(h.u(m).astype(np.float32)).cuda() for h in hist]
    v = [torch.from_numpy(h.v(m).astype(np.float32)).cuda() for h in hist]
    return u, v


@pytest.mark.parametrize("shape,lags,tile", [(None, None, 128), (3, 256, 128), (2, 64, 128),
                                             (5, 64, 128), (4, 1024, 128), (None, None, 64),
                                             (2, 64, 64), (4, 64, 64)])
def test_batch_equals_members_stepped_alone(shape, lags, tile):
    """Default launch (one CTA per 1024-lag item, pipeline shape 2) and others set with
    sbim_batch_set_conv_config, persistent (1-3) and one CTA per item (4-6), at 128
    and 64 orbit records per CTA (sbim_batch_set_conv_tile)."""
    from paper_2102_08756_gb300.sbim import SBIM
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        B, b, hist, dt = _setup(stream)
        if shape is not None:
            B.sbim_batch_set_conv_config(b, shape, lags)
        if tile != 128:
            B.sbim_batch_set_conv_tile(b, tile)
        alone = []
        for (a, c, n_cut, side) in MEMBERS:
            h = SBIM(a, c, a * 100.0, c * 100.0, CS, CP, RHO, dt, n_cut, side, "fp32", True,
                     stream=stream)
            h.set_conv_tile(tile)
            if shape is None:
                h.set_conv_config(2, 1024)
            else:
                h.set_conv_config(shape - 3 if shape > 3 else shape, lags)
            alone.append(h)
        oracles = [SBIMOracle(a, c, a * 100.0, c * 100.0, CS, CP, RHO, dt, n_cut, side)
                   for (a, c, n_cut, side) in MEMBERS[:2]]
        for m in range(60):
            u, v = _fields(hist, m)
            tau = [torch.empty_like(x) for x in u]
            B.sbim_batch_step(b, [x.data_ptr() for x in u], [x.data_ptr() for x in v],
                              [x.data_ptr() for x in tau])
            ref = [alone[k].step(u[k], v[k]) for k in range(len(MEMBERS))]
            stream.synchronize()
            for k in range(len(MEMBERS)):
                assert_finite(tau[k], "batched tau")
                assert torch.equal(tau[k], ref[k]), (m, k)
            for k, o in enumerate(oracles):
                r = o.step(u[k].double().cpu().numpy(), v[k].double().cpu().numpy())["tau"]
                got = tau[k].double().cpu().numpy()
                for c in range(3):
                    if np.linalg.norm(r[c]) > 0:
                        assert np.linalg.norm(got[c] - r[c]) / np.linalg.norm(r[c]) < 1e-5
        for h in alone:
            h.check()
            h.close()
        for k in range(len(MEMBERS)):
            B.sbim_check_device(B.sbim_batch_member(b, k))
        B.sbim_batch_destroy(b)


@pytest.mark.parametrize("shape,lags", [(None, None), (4, 1024), (5, 256)])
def test_bf16_batch_equals_members_stepped_alone(shape, lags):
    """Uncompensated BF16 hi-only history (SBIM_BF16, whose pipeline shapes are
    1-lag stages at 4 and 5 CTAs per SM): the default batch launch (persistent
    CTAs, shape 1, 1024-lag items) and one CTA per item (shapes 1 and 2) equal
    the members stepped alone with the same shape and lag chunking, bit for bit,
    and stay within the BF16 hi-only bound (1e-2) of the oracle."""
    from paper_2102_08756_gb300.sbim import SBIM
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        B, b, hist, dt = _setup(stream, precision=3, kahan=0)
        if shape is not None:
            B.sbim_batch_set_conv_config(b, shape, lags)
        alone = []
        for (a, c, n_cut, side) in MEMBERS:
            h = SBIM(a, c, a * 100.0, c * 100.0, CS, CP, RHO, dt, n_cut, side, "bf16", False,
                     stream=stream)
            if shape is None:
                h.set_conv_config(1, 1024)
            else:
                h.set_conv_config(shape - 3 if shape > 3 else shape, lags)
            alone.append(h)
        oracles = [SBIMOracle(a, c, a * 100.0, c * 100.0, CS, CP, RHO, dt, n_cut, side)
                   for (a, c, n_cut, side) in MEMBERS[:2]]
        for m in range(60):
            u, v = _fields(hist, m)
            tau = [torch.empty_like(x) for x in u]
            B.sbim_batch_step(b, [x.data_ptr() for x in u], [x.data_ptr() for x in v],
                              [x.data_ptr() for x in tau])
            ref = [alone[k].step(u[k], v[k]) for k in range(len(MEMBERS))]
            stream.synchronize()
            for k in range(len(MEMBERS)):
                assert_finite(tau[k], "batched tau")
                assert torch.equal(tau[k], ref[k]), (m, k)
            for k, o in enumerate(oracles):
                r = o.step(u[k].double().cpu().numpy(), v[k].double().cpu().numpy())["tau"]
                got = tau[k].double().cpu().numpy()
                for c in range(3):
                    if np.linalg.norm(r[c]) > 0:
                        assert np.linalg.norm(got[c] - r[c]) / np.linalg.norm(r[c]) < 1e-2
        for h in alone:
            h.check()
            h.close()
        for k in range(len(MEMBERS)):
            B.sbim_check_device(B.sbim_batch_member(b, k))
        B.sbim_batch_destroy(b)


def test_graph_replay_equals_direct_steps():
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        B, b1, hist, dt = _setup(stream)
        _, b2, _, _ = _setup(stream)
        ub = [torch.empty((3, c, a), device="cuda") for (a, c, _, _) in MEMBERS]
        vb = [torch.empty_like(x) for x in ub]
        tb = [torch.empty_like(x) for x in ub]
        B.sbim_batch_capture(b2, [x.data_ptr() for x in ub], [x.data_ptr() for x in vb],
                             [x.data_ptr() for x in tb])
        for m in range(50):
            u, v = _fields(hist, m)
            tau = [torch.empty_like(x) for x in u]
            B.sbim_batch_step(b1, [x.data_ptr() for x in u], [x.data_ptr() for x in v],
                              [x.data_ptr() for x in tau])
            for k in range(len(MEMBERS)):
                ub[k].copy_(u[k])
                vb[k].copy_(v[k])
            B.sbim_batch_replay(b2)
            stream.synchronize()
            for k in range(len(MEMBERS)):
                assert torch.equal(tau[k], tb[k]), (m, k)
        assert B.sbim_get_step(B.sbim_batch_member(b2, 0)) == 50
        B.sbim_batch_destroy(b1)
        B.sbim_batch_destroy(b2)


@pytest.mark.parametrize("shape,lags", [(None, None), (3, 16), (5, 16)])
def test_hybrid_ensemble_batch_and_graph(shape, lags):
    """Three coupled scenarios with different grids, slab thicknesses, fault laws
    and cutoffs: the ensemble step (one batched SBIM launch for the six
    half-spaces) and its CUDA-graph replay equal the scenarios stepped alone."""
    from paper_2102_08756_gb300 import sbim as B
    from paper_2102_08756_gb300.hybrid import Hybrid
    scen = [(16, 4, 16, 0.02, 30), (24, 6, 16, 0.05, 12), (32, 4, 24, 0.03, 45)]
    h = 100.0
    dt = 0.3 * h / CP
    stream = torch.cuda.Stream()

    def make():
        out = []
        for (n1, n2, n3, Dc, n_cut) in scen:
            x = Hybrid(n1, n2, n3, h, CS, CP, RHO, dt, n_cut, "fp32", True, True, stream=stream)
            i3, i1 = np.meshgrid(np.arange(n3), np.arange(n1), indexing="ij")
            patch = (np.abs(i1 - n1 / 2 + 0.5) < 3) & (np.abs(i3 - n3 / 2 + 0.5) < 3)
            x.set_fault(0.677, np.where(patch, 1.005 * 0.677 * 120e6, 70e6), 0.525, Dc, 120e6)
            out.append(x)
        return out

    with torch.cuda.stream(stream):
        alone, batched, graphed = make(), make(), make()
        for x in alone:
            _, _, top, bot = B.sbim_hybrid_info(x.h)
            single = 2 if shape is None else (shape - 3 if shape > 3 else shape)
            B.sbim_set_conv_config(top, single, lags or 1024)
            B.sbim_set_conv_config(bot, single, lags or 1024)
        b1 = B.sbim_hybrid_batch_create([x.h for x in batched])
        b2 = B.sbim_hybrid_batch_create([x.h for x in graphed])
        if shape is not None:
            B.sbim_hybrid_batch_set_conv_config(b1, shape, lags)
            B.sbim_hybrid_batch_capture(b2)                 # dropped by the next call
            B.sbim_hybrid_batch_set_conv_config(b2, shape, lags)
            with pytest.raises(B.SBIMError):
                B.sbim_hybrid_batch_replay(b2)
        B.sbim_hybrid_batch_capture(b2)
        for step in range(40):
            for x in alone:
                x.step()
            B.sbim_hybrid_batch_step(b1)
            B.sbim_hybrid_batch_replay(b2)
        stream.synchronize()
        for a, b, c in zip(alone, batched, graphed):
            ra, rb, rc = a.fault_fields()[1], b.fault_fields()[1], c.fault_fields()[1]
            ua, ub, uc = a.get_state()[0], b.get_state()[0], c.get_state()[0]
            stream.synchronize()
            assert torch.equal(ra, rb) and torch.equal(ra, rc)
            assert torch.equal(ua, ub) and torch.equal(ua, uc)
            assert float(ra.abs().max()) > 0.1
        B.sbim_hybrid_batch_destroy(b1)
        B.sbim_hybrid_batch_destroy(b2)
        for x in alone + batched + graphed:
            x.close()


def test_ensemble_members_at_full_size_equal_members_alone():
    """The ensemble configuration's own scenarios at their full sizes (the first
    four of the seeded draw the benchmark uses), in the benchmark's launch: the
    hybrid batch and its graph replay equal the scenarios stepped alone with the
    same lag chunking, bit for bit, over the first 25 steps of the rupture."""
    import bench
    from paper_2102_08756_gb300 import sbim as B
    from paper_2102_08756_gb300.hybrid import Hybrid
    scen = bench.ensemble_draw()[:4]
    h = 100.0
    dt = 0.3 * h / CP
    stream = torch.cuda.Stream()

    def make():
        out = []
        for sc in scen:
            n = sc["n"]
            x = Hybrid(n, sc["n2"], n, h, CS, CP, RHO, dt, sc["n_cut"], "fp32", True, True,
                       stream=stream)
            c = (np.arange(n) - n / 2 + 0.5) * h
            X3, X1 = np.meshgrid(c, c, indexing="ij")
            patch = (np.abs(X1) <= 1.5e3) & (np.abs(X3) <= 1.5e3)
            x.set_fault(0.677, np.where(patch, 1.005 * 0.677 * 120e6, sc["ratio"] * 0.677 * 120e6),
                        0.525, sc["Dc"], 120e6)
            out.append(x)
        return out

    with torch.cuda.stream(stream):
        alone, graphed = make(), make()
        for x in alone:
            _, _, top, bot = B.sbim_hybrid_info(x.h)
            B.sbim_set_conv_config(top, 2, 1024)
            B.sbim_set_conv_config(bot, 2, 1024)
        b = B.sbim_hybrid_batch_create([x.h for x in graphed])
        B.sbim_hybrid_batch_capture(b)
        for _ in range(25):
            for x in alone:
                x.step()
            B.sbim_hybrid_batch_replay(b)
        stream.synchronize()
        for a, g in zip(alone, graphed):
            assert torch.equal(a.fault_fields()[1], g.fault_fields()[1])
            assert torch.equal(a.get_state()[0], g.get_state()[0])
        assert max(float(x.fault_fields()[1].abs().max()) for x in alone) > 0.1
        B.sbim_hybrid_batch_destroy(b)
        for x in alone + graphed:
            x.close()
