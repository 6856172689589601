"""Checkpoint and restore of an SBIM handle (sbim_save / sbim_load): the state of
the truncated convolution of Eq. (SBI) is the step counter and the history ring;
a run restored from a checkpoint must continue bit-for-bit.  sbim_rewind takes
back one step: the next step re-evaluates that level."""
import numpy as np
import pytest

from paper_2102_08756_gb300.synth import separable_history

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CS, CP, RHO = 3464.0, 6000.0, 2670.0


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _make(n1, n3, n_cut, precision, side=1, dt=None):
    from paper_2102_08756_gb300.sbim import SBIM
    L = 100.0 * n1
    dt = dt or 0.3 * 100.0 / CP
    return SBIM(n1, n3, L, 100.0 * n3, CS, CP, RHO, dt, n_cut, side, precision, 1)


@pytest.mark.parametrize("precision", ["fp32", "fp64", "bf16x2", "bf16"])
@pytest.mark.parametrize("n_cut,split", [(7, 11), (24, 9)])
def test_restore_continues_bit_exact(precision, n_cut, split):
    n1, n3, steps = 24, 16, 20
    dt = 0.3 * 100.0 / CP
    hist = separable_history(n1, n3, 100.0 * n1, 100.0 * n3, steps, dt, CS, seed=7)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    a = _make(n1, n3, n_cut, precision)
    a.set_far_field((1.5e6, -2.0e6, 3.0e5))
    fields = [(torch.from_numpy(hist.u(m)).to("cuda", tdt), torch.from_numpy(hist.v(m)).to("cuda", tdt))
              for m in range(steps)]
    for m in range(split):
        a.step(*fields[m])
    ck = a.save()
    first = [a.step(*fields[m]).cpu().numpy() for m in range(split, steps)]

    b = _make(n1, n3, n_cut, precision)          # fresh handle, far field from the checkpoint
    b.load(ck)
    assert b.n == split
    second = [b.step(*fields[m]).cpu().numpy() for m in range(split, steps)]
    a.load(ck)                                   # the same handle, rewound
    third = [a.step(*fields[m]).cpu().numpy() for m in range(split, steps)]
    for x, y, z in zip(first, second, third):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_load_rejects_other_parameters_and_garbage():
    from paper_2102_08756_gb300.sbim import SBIMError
    a = _make(16, 16, 8, "fp32")
    z = torch.zeros((3, 16, 16), device="cuda")
    a.step(z, z)
    ck = a.save()
    for other in (_make(16, 16, 9, "fp32"), _make(16, 16, 8, "fp64"), _make(16, 16, 8, "fp32", side=-1),
                  _make(16, 16, 8, "fp32", dt=0.004), _make(16, 8, 8, "fp32")):
        with pytest.raises(SBIMError) as e:
            other.load(ck)
        assert e.value.code == -1
        assert other.n == 0
    bad = ck.copy()
    bad[0] ^= 0xFF
    with pytest.raises(SBIMError):
        a.load(bad)
    with pytest.raises(SBIMError):
        a.load(ck[:-1])
    assert a.n == 1
    from paper_2102_08756_gb300 import sbim
    import ctypes
    need = ctypes.c_size_t(0)
    sbim._check(sbim.lib().sbim_save(a.h, None, ctypes.byref(need)))
    small = np.empty(need.value - 1, dtype=np.uint8)
    cap = ctypes.c_size_t(small.nbytes)
    with pytest.raises(SBIMError):
        sbim._check(sbim.lib().sbim_save(a.h, small.ctypes.data, ctypes.byref(cap)))
    assert cap.value == need.value


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_rewind_reevaluates_the_level(precision):
    from paper_2102_08756_gb300.sbim import SBIMError
    n1, n3, n_cut = 16, 12, 6
    tdt = torch.float64 if precision == "fp64" else torch.float32
    g = torch.Generator().manual_seed(2)
    x = [torch.randn((3, n3, n1), generator=g, dtype=torch.float64).to("cuda", tdt) * 1e-3
         for _ in range(10)]
    a = _make(n1, n3, n_cut, precision)
    b = _make(n1, n3, n_cut, precision)
    with pytest.raises(SBIMError):
        a.rewind()
    for m in range(8):                     # past the cutoff: the ring has wrapped
        a.step(x[m], x[m + 1])
        b.step(x[m], x[m + 1])
    a.step(x[9], x[0])
    a.rewind()
    assert a.n == 8
    assert torch.equal(a.step(x[0], x[1]), b.step(x[0], x[1]))
    assert torch.equal(a.step(x[2], x[3]), b.step(x[2], x[3]))


@pytest.mark.parametrize("precision", ["fp32", "fp64", "bf16x2", "bf16"])
@pytest.mark.parametrize("variant,window", [(None, 0.0), (0, 0.0), (None, 3.0)])
def test_step_repeat_equals_rewind_and_step(precision, variant, window):
    """sbim_step_repeat re-evaluates the last level with a new displacement: the
    result matches sbim_rewind + sbim_step to rounding, and the ring slot it
    writes is the same, so every later step is bit-identical."""
    from paper_2102_08756_gb300.sbim import SBIMError
    n1, n3, n_cut = 20, 12, 7
    tdt = torch.float64 if precision == "fp64" else torch.float32
    g = torch.Generator().manual_seed(4)
    x = [torch.randn((3, n3, n1), generator=g, dtype=torch.float64).to("cuda", tdt) * 1e-3
         for _ in range(16)]
    a = _make(n1, n3, n_cut, precision)
    b = _make(n1, n3, n_cut, precision)
    for h in (a, b):
        if variant is not None:
            h.set_conv_config(variant)
        if window:
            h.set_window(window)
    with pytest.raises(SBIMError):
        a.step_repeat(x[0], x[1])
    for m in range(9):                               # past the cutoff
        a.step(x[m], x[m + 1])
        b.step(x[m], x[m + 1])
    a.step(x[9], x[10])
    b.step(x[9], x[10])
    ra = a.step_repeat(x[11], x[12])
    ra2 = a.step_repeat(x[13], x[14])                # a repeat can be repeated
    b.rewind()
    b.step(x[11], x[12])
    b.rewind()
    rb2 = b.step(x[13], x[14])
    assert a.n == b.n == 10
    tol = 1e-12 if precision == "fp64" else 1e-6
    scale = float(rb2.abs().max())
    assert float((ra2 - rb2).abs().max()) < tol * scale
    assert float((ra - ra2).abs().max()) > 0          # the new displacement mattered
    for m in range(3):
        assert torch.equal(a.step(x[m], x[m + 4]), b.step(x[m], x[m + 4]))
    a.rewind()
    with pytest.raises(SBIMError):
        a.step_repeat(x[0], x[1])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_coupled_rupture_restart_is_bit_exact(precision):
    """A coupled rupture (slab + slip-weakening fault + two half-spaces) saved
    mid-run and restored into a fresh handle continues bit-for-bit."""
    from paper_2102_08756_gb300.hybrid import Hybrid
    n, n2, h, n_cut = 24, 4, 100.0, 30
    dt = 0.3 * h / CP
    i3, i1 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    patch = (np.abs(i1 - n / 2 + 0.5) < 3) & (np.abs(i3 - n / 2 + 0.5) < 3)
    law = (np.full((n, n), 0.677), np.where(patch, 1.005 * 0.677 * 120e6, 70e6), 0.525, 0.02, 120e6)
    a = Hybrid(n, n2, n, h, CS, CP, RHO, dt, n_cut, precision)
    a.set_fault(*law)
    for _ in range(20):
        a.step()
    ck = a.save()
    ref = []
    for _ in range(25):                           # past the cutoff: the rings wrap
        a.step()
        ref.append(a.fault_fields()[1].cpu())
    b = Hybrid(n, n2, n, h, CS, CP, RHO, dt, n_cut, precision)
    b.set_fault(*law)
    b.load(ck)
    for r in ref:
        b.step()
        assert torch.equal(b.fault_fields()[1].cpu(), r)
    assert float(ref[-1].abs().max()) > 0.1


@pytest.mark.parametrize("symmetric", [False, True])
def test_fault_solver_restart_is_bit_exact(symmetric):
    from paper_2102_08756_gb300.fault import FaultSolver
    n, n_cut = 24, 30
    dt = 0.3 * 100.0 / CP
    i3, i1 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    patch = (np.abs(i1 - n / 2 + 0.5) < 3.5) & (np.abs(i3 - n / 2 + 0.5) < 3.5)
    law = (np.full((n, n), 0.677), np.where(patch, 1.005 * 0.677 * 120e6, 70e6), 0.525, 0.05, 120e6)
    a = FaultSolver(n, n, n * 100.0, n * 100.0, CS, CP, RHO, dt, n_cut, "fp32", symmetric)
    a.set_fault(*law)
    for _ in range(15):
        a.step()
    ck = a.save()
    ref = []
    for _ in range(25):
        a.step()
        ref.append(a.fault_fields()[1].cpu())
    b = FaultSolver(n, n, n * 100.0, n * 100.0, CS, CP, RHO, dt, n_cut, "fp32", symmetric)
    b.set_fault(*law)
    b.load(ck)
    for r in ref:
        b.step()
        assert torch.equal(b.fault_fields()[1].cpu(), r)
    assert float(ref[-1].abs().max()) > 0.1


@pytest.mark.parametrize("precision,rec_bytes", [("fp32", 32), ("fp64", 64)])
@pytest.mark.parametrize("variant", [2, 0])
def test_nan_canaries_in_padding_records_never_reach_the_output(precision, rec_bytes, variant):
    """NaN canaries in padding: the record tiles are padded to whole tiles of 128
    records whose member slots hold no Fourier bin.  A checkpoint whose ring
    holds NaN in every padding record, of every slot and component, is loaded;
    the following steps (the convolution reads those records every lag) give the
    same tractions, bit for bit, as a handle that never saw them.  Ring layout
    of one precision plane: [slot][component][record] records of 4 members."""
    from tests._layout import grid_records
    n1, n3, n_cut, split, steps = 16, 16, 12, 15, 25
    dt = 0.3 * 100.0 / CP
    hist = separable_history(n1, n3, 100.0 * n1, 100.0 * n3, steps, dt, CS, seed=9)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    fields = [(torch.from_numpy(hist.u(m)).to("cuda", tdt), torch.from_numpy(hist.v(m)).to("cuda", tdt))
              for m in range(steps)]
    a, b = _make(n1, n3, n_cut, precision), _make(n1, n3, n_cut, precision)
    for h in (a, b):
        h.set_conv_config(variant, 0)
    for m in range(split):
        a.step(*fields[m])
        b.step(*fields[m])
    ck = a.save()
    info = a.info()
    n_pad = info["n_slots"] // 4
    n_rec = len(grid_records(n1, n3, 100.0 * n1, 100.0 * n3)[0])
    assert n_pad > n_rec                                   # the grid has padding records
    head = ck.size - info["hist_bytes"]
    ring = ck[head:].view(np.float32 if precision == "fp32" else np.float64)
    ring = ring.reshape(n_cut, 3, n_pad, rec_bytes // ring.itemsize)
    ring[:, :, n_rec:, :] = np.nan
    a.load(ck)
    for m in range(split, steps):
        x = a.step(*fields[m]).cpu().numpy()
        y = b.step(*fields[m]).cpu().numpy()
        assert np.isfinite(x).all(), m
        assert np.array_equal(x, y), m
    a.check()
    b.check()
