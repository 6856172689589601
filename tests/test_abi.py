"""The C ABI library builds for sm_103a, loads without a GPU, exports every
entry point declared in include/sbim.h, and rejects invalid arguments before
touching the device."""
import os
import re

import pytest

from paper_2102_08756_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sbim.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sbim_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    from paper_2102_08756_gb300 import sbim
    return sbim.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sbim_create", "sbim_step", "sbim_destroy", "sbim_step_host",
                     "sbim_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_has_a_function_per_entry_point():
    from paper_2102_08756_gb300 import sbim
    for name in declared_functions():
        assert callable(getattr(sbim, name)), name


@pytest.mark.parametrize("args,msg", [
    (dict(n1=7), "even"),
    (dict(n3=0), "even"),
    (dict(cp=3000.0), "cp must exceed cs"),
    (dict(dt=0.0), "positive"),
    (dict(n_cut=0), "n_cut"),
    (dict(side=0), "side"),
    (dict(precision=9), "precision"),
])
def test_create_rejects_bad_arguments(lib, args, msg):
    from paper_2102_08756_gb300 import sbim
    kw = dict(n1=8, n3=8, L1=800.0, L3=800.0, cs=3464.0, cp=6000.0, rho=2670.0, dt=0.005,
              n_cut=8, side=1, precision=1, kahan=1, stream=None)
    kw.update(args)
    with pytest.raises(sbim.SBIMError) as e:
        sbim.sbim_create(**kw)
    assert e.value.code == -1
    assert msg in str(e.value)


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2102_08756_gb300 import sbim
    with pytest.raises(sbim.SBIMError):
        sbim.sbim_step(None, None, None, None)
    with pytest.raises(sbim.SBIMError):
        sbim.sbim_get_step(None)
    with pytest.raises(sbim.SBIMError):
        sbim.sbim_save(None)
    with pytest.raises(sbim.SBIMError):
        sbim.sbim_load(None, b"")
    sbim.sbim_destroy(None)


@pytest.mark.parametrize("kw,msg", [
    (dict(n1=7), "even"),
    (dict(cp=3000.0), "cp > cs"),
    (dict(dt=0.0), "dt"),
    (dict(precision=7), "precision"),
])
def test_fault_solver_rejects_bad_arguments(lib, kw, msg):
    from paper_2102_08756_gb300 import sbim
    a = dict(n1=8, n3=8, L1=800.0, L3=800.0, cs=3464.0, cp=6000.0, rho=2670.0, dt=0.005,
             n_cut=8, precision=1, symmetric=0, stream=None)
    a.update(kw)
    with pytest.raises(sbim.SBIMError) as e:
        sbim.sbim_fault_create(**a)
    assert e.value.code == -1 and msg in str(e.value)


@pytest.mark.parametrize("kw,msg", [
    (dict(n1=5), "even"),
    (dict(n2=3, fault=1), "n2"),
    (dict(cp=1000.0), "cp > cs"),
    (dict(precision=2), "SBIM_FP32 and SBIM_FP64"),
])
def test_hybrid_rejects_bad_arguments(lib, kw, msg):
    from paper_2102_08756_gb300 import sbim
    a = dict(n1=8, n2=4, n3=8, h=100.0, cs=3464.0, cp=6000.0, rho=2670.0, dt=0.005, n_cut=8,
             precision=1, boundaries=1, fault=1, stream=None)
    a.update(kw)
    with pytest.raises(sbim.SBIMError) as e:
        sbim.sbim_hybrid_create(**a)
    assert e.value.code == -1 and msg in str(e.value)


def test_null_handles_of_the_other_objects_fail_cleanly(lib):
    from paper_2102_08756_gb300 import sbim
    for call, args in ((sbim.sbim_fault_step, (None,)), (sbim.sbim_hybrid_step, (None,)),
                       (sbim.sbim_batch_set_conv_config, (None, 1, 0)),
                       (sbim.sbim_hybrid_batch_set_conv_config, (None, 1, 0)),
                       (sbim.sbim_rewind, (None,)), (sbim.sbim_step_repeat, (None, None, None, None)),
                       (sbim.sbim_selftest_wait_timeout, (None,))):
        with pytest.raises(sbim.SBIMError) as e:
            call(*args)
        assert e.value.code == -1
    sbim.sbim_fault_destroy(None)
    sbim.sbim_hybrid_destroy(None)
    sbim.sbim_batch_destroy(None)
