"""GPU: run-time instability detection.  A non-finite value written into a
field from the host (the failure is made on the host; no GPU fault is involved)
must be found by fdtd_check_finite and by the periodic check inside
fdtd_step, reported as FDTD_EUNSTABLE once, and leave the context usable."""
import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from tests._helpers import assert_fields_close, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_check_finite_finds_a_nan_written_from_the_host():
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=160, nsteps=40, npml=12)
    sim = fdtd.from_scene(sc)
    sim.step(40)
    sim.check_finite()                         # a normal run is finite
    hy = sim.get_field("hy", (sc.ny, sc.nx))
    hy[77, 91] = np.nan
    sim.set_field("hy", hy)
    with pytest.raises(fdtd.FDTDError) as ei:
        sim.check_finite()
    assert ei.value.code == fdtd.EUNSTABLE
    sim.close()


@pytest.mark.parametrize("kernel", [0, 1])
def test_periodic_check_reports_a_blow_up_once(kernel):
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=160, nsteps=64, npml=12)
    sim = fdtd.from_scene(sc)
    sim.set_option("kernel", kernel)
    sim.set_option("check_every", 8)
    assert sim.get_option("check_every") == 8
    sim.step(64)
    sim.sync()                                  # finite: nothing reported
    assert_fields_close({c: sim.get_field(c, (sc.ny, sc.nx)) for c in ("ez", "hx", "hy")}, oracle_run(sc, 64))
    ez = sim.get_field("ez", (sc.ny, sc.nx))
    ez[40, 50] = np.inf
    sim.set_field("ez", ez)
    sim.step(12)                                # passes step 72: the scan runs
    with pytest.raises(fdtd.FDTDError) as ei:
        sim.sync()
    assert ei.value.code == fdtd.EUNSTABLE
    sim.sync()                                  # reported once
    sim.reset()
    sim.step(64)
    sim.sync()                                  # the context is usable again
    sim.close()


def test_check_finite_3d():
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.box_scene(side=32, nsteps=10, npml=4, n_boxes=4)
    sim = fdtd.from_scene(sc)
    sim.step(10)
    sim.check_finite()
    hz = sim.get_field("hz", (sc.nz, sc.ny, sc.nx))
    hz[5, 6, 7] = np.nan
    sim.set_field("hz", hz)
    with pytest.raises(fdtd.FDTDError) as ei:
        sim.check_finite()
    assert ei.value.code == fdtd.EUNSTABLE
    with pytest.raises(fdtd.FDTDError):
        sim.set_option("check_every", 4)        # the periodic check covers 2D contexts
    sim.close()
