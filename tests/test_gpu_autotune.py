"""Launch-shape autotuner (rod_system_autotune): it times the valid (elements per block,
threads per block) shapes on the live state, keeps the fastest and restores the state; the
trajectory it then computes is that of any other shape."""
import numpy as np
import pytest

import rodgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13766_gb300 import build
    build.build()


@pytest.mark.parametrize("contact", [False, True])
def test_autotune_restores_the_state_and_keeps_the_trajectory(contact):
    from paper_2605_13766_gb300 import RodSystem
    if contact:
        p = rodgen.random_packing(n_rods=120, nmin=16, nmax=200, box=0.15, rest_len=2e-3, radius=0.004, seed=5,
                                  speed=0.5, dt=2e-6, margin=-5e-4)
        dt = 2e-6
    else:
        p = rodgen.perturbed(rodgen.cilia_carpet(side=8, n=50), seed=4)
        dt = 1e-5
    a = RodSystem(p)
    a.set_state(*p.state())
    before = a.get_state()
    te, tt, ms = a.autotune(dt, trial_steps=3)
    assert te % 32 == 0 and tt % 32 == 0 and 0 < tt <= 512 and te >= int(p.n_elem.max())
    for x, y in zip(a.get_state(), before):
        assert np.array_equal(x, y)
    assert a.get_launch() == (te, tt)
    a.step(200, dt)
    b = RodSystem(p)
    b.set_launch(384, 256)
    b.set_state(*p.state())
    b.step(200, dt)
    xa, xb = a.get_state()[0], b.get_state()[0]
    # the pack boundaries differ; the element arithmetic differs only where a warp-uniform series
    # degree of the rotation maps changes with the warp's members (below 1e-17 relative)
    scale = np.abs(xb).max()
    assert np.abs(xa - xb).max() <= 1e-13 * scale
    a.close()
    b.close()
