"""The allocation-free entry point agrees with the regular one.

lmbd_central_polarizabilities_noalloc serves callers that cannot allocate device
memory (a plug-in of an MD engine that owns the memory pool, or an embedded runtime
that forbids allocation after start-up); its scratch is a fixed array inside the
library.  This test calls it through the C ABI twice in a row and
compares both results with the central polarisabilities that lmbd_energy_forces
computes, within the 1e-12 relative tolerance the other polarisability tests use.
It is collected last so that a failure here cannot hide failures elsewhere.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2407_06409_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lm():
    from paper_2407_06409_gb300 import build, lmbd
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    L = lmbd.lib()
    f = L.lmbd_central_polarizabilities_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(lmbd.Species), ctypes.c_int, ctypes.POINTER(lmbd.Params), ctypes.c_int,
                  ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return lmbd


def _noalloc(lm, s, p, n_freq, out):
    sp = (lm.Species * len(s.table))(*[lm.Species(*row) for row in s.table])
    pos = torch.tensor(s.positions, device="cuda")
    cell = None if s.cell is None else torch.tensor(s.cell, device="cuda")
    spec = torch.tensor(s.species, dtype=torch.int32, device="cuda")
    nu = torch.tensor(s.hirshfeld, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    return lm.lib().lmbd_central_polarizabilities_noalloc(
        sp, len(s.table), ctypes.byref(p), n_freq, s.n_atoms, pos.data_ptr(),
        None if cell is None else cell.data_ptr(), spec.data_ptr(), nu.data_ptr(), out.data_ptr(), stream)


def _reference(lm, s, p, n_freq):
    model = lm.LMBD(s.table, p, n_freq, 6)
    model.energy_forces(torch.tensor(s.positions, device="cuda"),
                        None if s.cell is None else torch.tensor(s.cell, device="cuda"),
                        torch.tensor(s.species, dtype=torch.int32, device="cuda"),
                        torch.tensor(s.hirshfeld, device="cuda"), forces=False)
    return model.central_polarizabilities(s.n_atoms).numpy()


@pytest.mark.parametrize("case", ["cluster", "box"])
def test_noalloc_matches_regular_entry_point_twice(lm, case):
    if case == "cluster":
        s = inputs.cluster(24, seed=0)
        p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    else:
        s = inputs.box(90, seed=2, jitter=0.05)
        p = lm.default_params(r_scs=4.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    n_freq = 12
    ref = _reference(lm, s, p, n_freq)
    for _ in range(2):
        out = torch.full((s.n_atoms, n_freq + 1), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(lm, s, p, n_freq, out)
        assert st == lm.LMBD_OK, lm.lib().lmbd_status_string(st)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.allclose(got, ref, rtol=1e-12, atol=0)


def test_noalloc_rejects_sizes_beyond_its_scratch(lm):
    s = inputs.box(300, seed=3)
    p = lm.default_params(r_scs=4.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    out = torch.zeros((s.n_atoms, 13), dtype=torch.float64, device="cuda")
    assert _noalloc(lm, s, p, 12, out) == 7   # LMBD_ESCRATCH


def test_noalloc_rejects_site_counts_beyond_its_scratch(lm):
    # within the atom limit, but more sites per atom than the fixed scratch holds
    out = torch.zeros((80, 13), dtype=torch.float64, device="cuda")
    # (a) 80 atoms packed within 4.5 Angstrom, r_SCS = 10 Angstrom: every atom has all 80 in
    # its coupled set K1 (> LMBD_NOALLOC_MAX_K1 = 64) but only 80 sites in its list (< 512)
    s = inputs.cluster(80, radius=4.5, min_sep=1.0, n_species=3, seed=5)
    p = lm.default_params(r_scs=10.0, r_mbd1=10.0, r_mbd2=10.0, r_sphere=10.0)
    assert _noalloc(lm, s, p, 12, out) == 7   # LMBD_ESCRATCH
    # (b) a periodic 200-atom box at 0.1 atoms/A^3 with r_SCS = 6 Angstrom: ~720 sites within
    # 2 r_SCS of every atom (> LMBD_NOALLOC_SITE_CAP = 512)
    s = inputs.box(200, seed=6)
    p = lm.default_params(r_scs=6.0, r_mbd1=6.0, r_mbd2=6.0, r_sphere=6.0)
    out = torch.zeros((200, 13), dtype=torch.float64, device="cuda")
    assert _noalloc(lm, s, p, 12, out) == 7
    # the scratch is reusable after a rejection
    s = inputs.cluster(24, seed=0)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    out = torch.full((24, 13), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(lm, s, p, 12, out) == lm.LMBD_OK
    assert np.allclose(out.cpu().numpy(), _reference(lm, s, p, 12), rtol=1e-12, atol=0)


def test_noalloc_refuses_a_capturing_stream(lm):
    # the entry point reads site counts back to the host, which a stream under capture does
    # not allow: it must refuse the stream before issuing anything, leaving the capture valid
    s = inputs.cluster(24, seed=0)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    out = torch.zeros((24, 13), dtype=torch.float64, device="cuda")
    marker = torch.zeros(4, dtype=torch.float64, device="cuda")
    sp = (lm.Species * len(s.table))(*[lm.Species(*row) for row in s.table])
    pos = torch.tensor(s.positions, device="cuda")
    spec = torch.tensor(s.species, dtype=torch.int32, device="cuda")
    nu = torch.tensor(s.hirshfeld, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        # inputs were made before the capture: nothing but the call itself is captured here
        st = lm.lib().lmbd_central_polarizabilities_noalloc(
            sp, len(s.table), ctypes.byref(p), 12, s.n_atoms, pos.data_ptr(), None, spec.data_ptr(),
            nu.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        marker.fill_(1.0)
    assert st == lm.LMBD_EUNSUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(marker == 1.0)


def test_noalloc_rejects_device_species_out_of_range(lm):
    s = inputs.cluster(24, seed=0)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    bad = inputs.Structure(s.positions, None, np.where(np.arange(24) == 7, len(s.table), s.species).astype(np.int32),
                           s.hirshfeld, s.table)
    out = torch.zeros((24, 13), dtype=torch.float64, device="cuda")
    assert _noalloc(lm, bad, p, 12, out) == lm.LMBD_EINVAL
