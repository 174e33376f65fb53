"""Autotuner of the SCS launch shapes (lmbd_autotune): picks a bucket width from its
candidate set by timing, keeps it in the context, and changes no result."""
import pytest
import torch

from paper_2407_06409_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lm():
    from paper_2407_06409_gb300 import build, lmbd
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lmbd


def _dev(s):
    return (torch.tensor(s.positions, device="cuda"), torch.tensor(s.cell, device="cuda"),
            torch.tensor(s.species, dtype=torch.int32, device="cuda"), torch.tensor(s.hirshfeld, device="cuda"))


def test_autotune_picks_a_width_and_keeps_results(lm):
    s = inputs.box(512, seed=0)
    model = lm.LMBD(s.table, lm.default_params(), 12, 6)
    e0, f0 = model.energy_forces(*_dev(s), forces=True)
    w = model.autotune(*_dev(s))
    assert w in (2, 3, 4, 6, 8, 12, 16)
    e1, f1 = model.energy_forces(*_dev(s), forces=True)
    assert torch.equal(e0, e1)
    assert (f0 - f1).abs().max().item() < 1e-12
    # per-atom launch mode has no buckets to tune
    model.set_launch_mode(lm.LAUNCH_PER_ATOM)
    with pytest.raises(lm.LmbdError) as err:
        model.autotune(*_dev(s))
    assert err.value.status == lm.LMBD_EINVAL
