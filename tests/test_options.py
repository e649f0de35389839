"""Argument checks of fams_setup_batch on the CPU: every invalid grid,
fracture or option value is rejected with FAMS_EINVAL and its reason before
any CUDA call, so these run without a GPU (and give the same answers with
one)."""
import copy

import numpy as np
import pytest

from paper_1705_05784_gb300 import inputs


def _fams():
    from paper_1705_05784_gb300 import build
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(f"no CUDA toolkit: {e}")
    from paper_1705_05784_gb300 import fams
    return fams


def _set(**kw):
    def f(p):
        for k, v in kw.items():
            setattr(p, k, v)
    return f


CASES = [
    ("dim", _set(dim=4), "grid.dim must be 2 or 3"),
    ("nx", _set(nx=0), "grid sizes must be >= 1"),
    ("dx", _set(dx=0.0), "cell sizes must be > 0"),
    ("no Dirichlet face", _set(bc_mask=0), "at least one Dirichlet face is required"),
    ("aperture", _set(aperture=0.0), "aperture and h_f must be > 0"),
    ("coarsening", _set(coarsen=(0, 4, 1)), "coarsening ratios must be >= 1"),
    ("basis", _set(basis=4), "basis must be 0..3"),
    ("restriction", _set(restriction=3), "restriction must be"),
    ("alpha = 1", _set(alpha=1.0), "alpha must be in [0, 1)"),
    ("alpha < 0", _set(alpha=-0.1), "alpha must be in [0, 1)"),
    ("max_iter", _set(max_iter=-1), "max_iter must be >= 0"),
    ("precision", _set(precision=2), "precision must be"),
    ("krylov", _set(krylov=2), "krylov must be"),
    ("restart 0", _set(krylov=1, restart=0), "GMRES restart must be in 1..FAMS_MAX_RESTART"),
    ("restart too long", _set(krylov=1, restart=100000), "GMRES restart must be in"),
    ("prepare_flux", _set(prepare_flux=2), "prepare_flux must be 0 or 1"),
    ("merge_cap", _set(merge_cap=-1), "merge_cap must be >= 0"),
    ("grid_solve", _set(grid_solve=2), "grid_solve must be -1, 0 or 1"),
    ("subblock", _set(subblock=2), "subblock must be 0 or 1"),
    ("subblock + mixed", _set(subblock=1, precision=1), "subblock needs precision FAMS_FP64"),
    ("bf16_p", _set(bf16_p=2, precision=1), "bf16_p must be 0 or 1"),
    ("bf16_p + FP64", _set(bf16_p=1), "bf16_p needs precision FAMS_MIXED"),
    ("coarse_mode", _set(coarse_mode=3), "coarse_mode must be 0, 1 or 2"),
]


@pytest.mark.parametrize("name,change,reason", CASES, ids=[c[0] for c in CASES])
def test_invalid_setup_is_rejected_before_any_cuda_call(name, change, reason):
    fams = _fams()
    p = copy.deepcopy(inputs.config_2d_small())
    change(p)
    with pytest.raises(fams.FamsError) as e:
        fams.Context(p)
    assert e.value.status == fams.EINVAL, str(e.value)
    assert reason in str(e.value), str(e.value)


def test_an_invalid_instance_rejects_the_whole_batch():
    """A batch is checked instance by instance before anything is allocated:
    one bad instance among good ones fails the setup with its reason."""
    fams = _fams()
    good = inputs.config_2d_small()
    bad = copy.deepcopy(good)
    bad.coarsen = (4, 0, 1)
    with pytest.raises(fams.FamsError) as e:
        fams.Context([good, good, bad])
    assert e.value.status == fams.EINVAL
    assert "coarsening ratios must be >= 1" in str(e.value)


def test_3d_plate_arrays_are_checked():
    fams = _fams()
    p = inputs.config_3d(12, 12, 8, 1.0, (4, 4, 2), 2, (4, 8), 1e3, (4, 4, 4), 4, 4, seed=3)
    assert p.fracs is not None and len(p.fracs) > 0
    p.h_f = -1.0
    with pytest.raises(fams.FamsError) as e:
        fams.Context(p)
    assert e.value.status == fams.EINVAL
    assert "aperture and h_f must be > 0" in str(e.value)
    assert np.all(np.isfinite(p.perm))
