"""cgevap_calibrate_threshold on the paper's flat interface (Sec. III.A.1: D3Q19 4x128x4, walls at
the y ends, beta = 0.99, sigma = 0.1, S-bar = 3, phi = 0.03): the calibrated Gamma lies between the
paper's 0.305 and 0.31, and the oracle measures the same S-bar at it."""
import pytest

import oracle
from paper_2412_14859_gb300.binding import SITES_GRADIENT, calibrate_threshold
from test_oracle_paper_benchmarks import flat_run, mean_sbar

pytestmark = pytest.mark.gpu


def test_calibrated_gamma_on_flat_interface():
    thr, sb = calibrate_threshold(19, 4, 128, 4, periodic=(1, 0, 1), phi=0.03, target_sbar=3.0,
                                  sigma=0.1, beta=0.99, site_rule=SITES_GRADIENT, storage="f64")
    assert 0.305 <= thr <= 0.31
    assert sb == pytest.approx(3.0, abs=0.02)
    p, run = flat_run(thr)
    assert mean_sbar(p, run, thr) == pytest.approx(sb, abs=1e-3)


def test_calibration_rejects_bad_arguments():
    from paper_2412_14859_gb300.binding import CgevapError
    with pytest.raises(CgevapError, match="ARG"):
        calibrate_threshold(19, 4, 128, 4, phi=-1.0)
    with pytest.raises(CgevapError, match="ARG"):
        calibrate_threshold(19, 4, 8, 4, phi=0.03)
    with pytest.raises(CgevapError, match="UNSUPPORTED"):
        calibrate_threshold(19, 4, 128, 4, phi=0.03, storage="f16dev")
