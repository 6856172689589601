"""Host planning of the spectral layout (include/sbim.h, sbim_plan), without a
GPU: the orbit records group the half-spectrum bins by exact |k| (the kernel
arguments T = m |k| c_s dt of Section 2.3 are shared within a record), checked
against rational-arithmetic grouping; the history size follows the record size
of each precision; invalid grids are rejected."""
import pytest

from paper_2102_08756_gb300 import _build
from tests._layout import _classes, expected_slots, grid_records

REC_BYTES = {"fp64": 64, "fp32": 32, "bf16x2": 32, "bf16": 16}


@pytest.fixture(scope="module")
def plan():
    _build.build()
    from paper_2102_08756_gb300.sbim import sbim_plan
    return sbim_plan


@pytest.mark.parametrize("n1,n3,L1,L3", [
    (64, 64, 6400.0, 6400.0),      # square: classes {(a,b),(a,-b),(b,a),(b,-a)}
    (16, 12, 1600.0, 1200.0),      # L1/L3 = 4/3
    (64, 32, 6400.0, 3200.0),      # equal spacings, L1/L3 = 2
    (48, 32, 4800.0, 3200.0),      # L1/L3 = 3/2
    (40, 24, 4000.0, 2520.3),      # no small fraction: floating-point grouping
    (2, 6, 200.0, 600.0),          # degenerate: k1 = 0 or Nyquist only
    (6, 2, 600.0, 200.0),
])
def test_slots_match_exact_wavenumber_classes(plan, n1, n3, L1, L3):
    p = plan(n1, n3, L1, L3, 8, "fp32")
    assert p["n_modes"] == n3 * (n1 // 2 + 1)
    assert p["n_slots"] == expected_slots(n1, n3, L1, L3)


def test_tpv3_plane_and_square_headline_grid(plan):
    # the 1024 x 512 plane of the TPV3 runs (dx = 50 m): whole records would take
    # 314,568 slots (1.20x the bins, most classes being pairs); half records
    # take 264,704 with the tile padding (1.008x)
    p = plan(1024, 512, 51200.0, 25600.0, 1600, "fp32")
    assert p["n_modes"] == 262656 and p["n_slots"] == 264704
    assert p["n_slots"] <= 1.03 * p["n_modes"]
    # the 1024^2 boundary with a 4096-lag FP32 history: 52.04 GB
    q = plan(1024, 1024, 102400.0, 102400.0, 4096, "fp32")
    assert q["n_slots"] == 529408 and q["hist_bytes"] == 52042924032


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x2", "bf16"])
def test_history_bytes_per_precision(plan, precision):
    n_cut = 37
    p = plan(32, 24, 3200.0, 2400.0, n_cut, precision)
    assert p["hist_bytes"] == n_cut * 3 * (p["n_slots"] // 4) * REC_BYTES[precision]


@pytest.mark.parametrize("args", [
    (7, 8, 700.0, 800.0, 4, "fp32"),
    (8, 0, 800.0, 800.0, 4, "fp32"),
    (8, 8, 0.0, 800.0, 4, "fp32"),
    (8, 8, 800.0, 800.0, 0, "fp32"),
    (8, 8, 800.0, 800.0, 4, 9),
])
def test_plan_rejects_bad_arguments(plan, args):
    from paper_2102_08756_gb300.sbim import SBIMError
    with pytest.raises(SBIMError):
        plan(*args)


@pytest.mark.parametrize("n1,n3,L1,L3", [(16, 12, 1600.0, 1200.0), (64, 32, 6400.0, 3200.0),
                                        (32, 32, 3200.0, 3200.0), (384, 384, 38400.0, 38400.0),
                                        (6, 2, 600.0, 200.0)])
def test_layout_model_is_a_partition(n1, n3, L1, L3):
    """The record model the tests compare with: every bin in exactly one record,
    at most 4 member slots per record, at most two |k| per record (one per
    half), whole records (one |k| each) on the square grids and half records on
    the rectangular planes."""
    records, halves = grid_records(n1, n3, L1, L3)
    nh = n1 // 2 + 1
    slots = {}
    key = {}
    for k, cls in enumerate(_classes(n1, n3, L1, L3)):
        for flat, s_ in cls:
            slots[flat] = s_
            key[flat] = k
    seen = [b for rec in records for b in rec]
    assert sorted(seen) == list(range(n3 * nh))
    for rec in records:
        assert sum(slots[b] for b in rec) <= 4
        assert len({key[b] for b in rec}) <= (2 if halves else 1)
    assert halves == (n1 != n3 and L1 != L3)
