"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function the header declares, and rejects bad arguments before touching
the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2603_03639_gb300 import build, tnrc
    if not os.path.exists(tnrc.LIB_PATH):
        build.build()
    return tnrc.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tnrc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tnrc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tnrc_create", "tnrc_set_controls", "tnrc_sample_noise", "tnrc_fidelity", "tnrc_fidelity_grad"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    from paper_2603_03639_gb300 import tnrc
    names = declared_functions()
    assert set(names) == set(tnrc.EXPORTS)
    for n in names:
        assert getattr(L, n) is not None


def test_status_strings(L):
    for s in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.tnrc_status_string(s)
        assert b"unknown" not in L.tnrc_status_string(s)
    assert b"unknown" in L.tnrc_status_string(42)


def test_create_rejects_bad_arguments_without_a_device(L):
    from paper_2603_03639_gb300 import tnrc
    import synth
    ins = synth.product_inputs(4, 1, 0)
    base = dict(N=4, K=2, dt=0.1, chi=4, M=1, C=2)
    bad = [dict(base, N=1), dict(base, K=0), dict(base, chi=0), dict(base, chi=65), dict(base, dt=-1.0),
           dict(base, M=0), dict(base, C=4)]
    dims, data = tnrc._pack(ins[0])
    good = (tnrc.MPSDesc * 2)()
    for x in good:
        x.n_sites = 4
        x.bond_dims = dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        x.data = data.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    tg = ctypes.cast(ctypes.byref(good, ctypes.sizeof(tnrc.MPSDesc)), ctypes.POINTER(tnrc.MPSDesc))
    for kw in bad:
        pb, keep = tnrc.make_problem(kw["N"], kw["K"], kw["dt"], kw["chi"], kw["M"], kw["C"], 1)
        h = ctypes.c_void_p()
        st = L.tnrc_create(ctypes.byref(pb), good, tg, None, ctypes.byref(h))
        assert st == -1, kw
        assert not h.value
    # null arguments
    pb, keep = tnrc.make_problem(4, 2, 0.1, 4, 1, 2, 1)
    assert L.tnrc_create(None, None, None, None, None) == -1
    h = ctypes.c_void_p()
    assert L.tnrc_create(ctypes.byref(pb), None, None, None, ctypes.byref(h)) == -1
    # an MPS of the wrong length or with a bad boundary bond
    dims = np.array([1, 1, 1, 1], dtype=np.int32)
    data = np.zeros(2 * 2 * 3)
    d = (tnrc.MPSDesc * 2)()
    for x in d:
        x.n_sites = 3
        x.bond_dims = dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        x.data = data.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.tnrc_create(ctypes.byref(pb), d, ctypes.cast(ctypes.byref(d, ctypes.sizeof(tnrc.MPSDesc)),
                                                          ctypes.POINTER(tnrc.MPSDesc)), None, ctypes.byref(h)) == -1
    # the struct size guards against a mismatched header
    pb.struct_size = 8
    assert L.tnrc_create(ctypes.byref(pb), d, d, None, ctypes.byref(h)) == -1


def test_null_context_calls_are_rejected(L):
    dp = ctypes.POINTER(ctypes.c_double)
    x = np.zeros(4)
    assert L.tnrc_set_controls(None, x.ctypes.data_as(dp), 4) == -1
    assert L.tnrc_sample_noise(None, 1, 0, 0.1) == -1
    assert L.tnrc_set_noise(None, x.ctypes.data_as(dp), 4) == -1
    assert L.tnrc_fidelity(None, x.ctypes.data_as(dp), None) == -1
    assert L.tnrc_fidelity_grad(None, x.ctypes.data_as(dp), x.ctypes.data_as(dp)) == -1
    assert L.tnrc_sync(None) == -1
    L.tnrc_destroy(None)


def test_footprint_grows_with_the_problem(L):
    from paper_2603_03639_gb300 import tnrc
    small = tnrc.footprint(8, 20, 0.05, 16, 16, 2, 4)
    big = tnrc.footprint(50, 100, 0.05, 64, 256, 3, 8)
    assert 0 < small < big
    assert tnrc.footprint(1, 20, 0.05, 16, 16, 2, 4) == 0


def test_discretisation_and_form_fields_are_validated(L):
    """trotter_order, substeps, operator_form, crosstalk_terms and the launch
    shape are checked on the host: a bad value gives a zero footprint (and
    TNRC_E_INVALID from tnrc_create) before any device call."""
    from paper_2603_03639_gb300 import tnrc
    args = (8, 20, 0.05, 16, 16, 3, 4)
    assert tnrc.footprint(*args) > 0
    for kw in (dict(order=3), dict(order=-1), dict(substeps=-1), dict(crosstalk=2), dict(ctas_per_sm=9),
               dict(warps=9), dict(warps=1)):
        assert tnrc.footprint(*args, **kw) == 0, kw
    pb, _ = tnrc.make_problem(*args)
    pb.operator_form = 2
    assert L.tnrc_footprint(ctypes.byref(pb)) == 0
    # operators: theta is 4 chi wide, so chi is capped at 32
    assert tnrc.footprint(8, 20, 0.05, 32, 16, 3, 1, operator=True) > 0
    assert tnrc.footprint(8, 20, 0.05, 33, 16, 3, 1, operator=True) == 0


def test_footprint_follows_the_discretisation_and_form(L):
    """More truncated layers (first order: 2 per step; substeps) and the
    operator form's wider sites need more memory."""
    from paper_2603_03639_gb300 import tnrc
    args = (10, 20, 0.05, 16, 16, 3, 2)
    base = tnrc.footprint(*args)
    assert tnrc.footprint(*args, substeps=3) > base
    assert tnrc.footprint(*args, operator=True) > base
    assert tnrc.footprint(*args, order=1) > 0


def _static_case(w):
    from oracle import noise
    ins, tgs = w.states()
    J = noise.sample_J(w.seed_J, w.M, w.N, w.noise_dist, w.noise_scale, terms=w.crosstalk)
    return ins, tgs, w.controls(), J, w.mask()


def test_static_entry_validates_on_the_host(L):
    """tnrc_fidelity_static checks the problem, its arrays and its size
    against the static array on the host, before any device call: an
    oversize problem is TNRC_E_TOO_LARGE, non-finite controls, noise or
    fixed couplings TNRC_E_INVALID, on a machine with or without a GPU."""
    from paper_2603_03639_gb300 import tnrc
    import synth
    w = synth.WORKLOADS["cnot50"].replace(M=64)
    ins, tgs, u, J, mask = _static_case(w)
    with pytest.raises(tnrc.TNRCError) as e:
        tnrc.fidelity_static(w.N, w.K, w.dt, w.chi, w.C, ins, tgs, u, J, mask=mask)
    assert e.value.status == -7
    w = synth.WORKLOADS["x8"].replace(M=2)
    ins, tgs, u, J, mask = _static_case(w)
    for bad_u, bad_J, gfix in ((np.where(np.arange(u.size).reshape(u.shape) == 5, np.nan, u), J, None),
                               (u, np.where(np.arange(J.size).reshape(J.shape) == 3, np.inf, J), None),
                               (u, J, np.full((w.K, w.N - 1), np.inf))):
        with pytest.raises(tnrc.TNRCError) as e:
            tnrc.fidelity_static(w.N, w.K, w.dt, w.chi, w.C, ins, tgs, bad_u, bad_J, mask=mask, g_fixed=gfix)
        assert e.value.status == -1


def test_static_entry_without_a_device_reports_cuda_error(L):
    """A valid problem on a machine without a GPU: TNRC_E_CUDA, no crash."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2603_03639_gb300 import tnrc
    import synth
    w = synth.WORKLOADS["x8"].replace(M=2)
    ins, tgs, u, J, mask = _static_case(w)
    with pytest.raises(tnrc.TNRCError) as e:
        tnrc.fidelity_static(w.N, w.K, w.dt, w.chi, w.C, ins, tgs, u, J, mask=mask)
    assert e.value.status == -3
