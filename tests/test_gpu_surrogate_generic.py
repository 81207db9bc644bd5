"""The surrogate's runtime-width kernel paths (rows S1-S4 for species and element counts the
fixed-size instances do not cover).  The H2 mechanism with an inert argon appended has 10 species
and 4 elements: its forward pass runs the runtime-width instance of the fused network kernel and
its post-processing the general kernel (the 9-species, 3-element instances serve the H2 model).
Both are compared with the oracle exactly as the fixed-size instances are."""
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import surrogate as osur  # noqa: E402

from helpers import random_states, with_inert_argon  # noqa: E402
from test_gpu_surrogate import check_forward_against_oracle  # noqa: E402
from test_gpu_surrogate_post import _compare, _params  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h2_ar(h2):
    m = with_inert_argon(h2)
    assert (m.ns, m.ne) == (10, 4)
    return m


@pytest.fixture(scope="module")
def om_h2_ar(h2_ar):
    return oracle.OracleMech(h2_ar)


@pytest.mark.parametrize("n", [1000, 152 * 128 + 77])
def test_forward_runtime_width_matches_oracle(h2_ar, n):
    """Network output, trust box and inverse transform of the runtime-width instance; the second
    size gives some CTAs a second tile."""
    check_forward_against_oracle(h2_ar, n)


def test_post_general_elementwise_vs_oracle(h2_ar, om_h2_ar):
    """Projection (four elements) and Newton on T of the general post-processing kernel against
    the oracle on the device's network output, cell by cell; the route of every cell as the
    oracle decides; the fallback cells bitwise the FP64 integrator's result."""
    T, p, Y = random_states(h2_ar, 2000, 53, "H2", Tlo=600.0, Thi=2400.0)
    prm = _params(h2_ar, osur.features(T, p, Y), 63, out_scale=1.0, y_std=0.05)
    why, n_net, n_near = _compare(h2_ar, om_h2_ar, prm, T, p, Y)
    assert n_net >= 1900, (why, n_net)
    assert n_near <= 5


def test_post_general_failures_fall_back(h2_ar, om_h2_ar):
    """Large composition changes and states outside the Newton range take the FP64 route in the
    general kernel as the oracle decides (with this network and these states 3 cells fail the
    conservation test and 134 the Newton test; the route of every cell is compared)."""
    T, p, Y = random_states(h2_ar, 1500, 54, "H2", Tlo=800.0, Thi=2400.0)
    T[:6] = 150.0
    T[6:12] = 6500.0
    prm = _params(h2_ar, osur.features(T, p, Y), 64, out_scale=3.0, y_std=3.0)
    prm["box_lo"][0] = 100.0
    prm["box_hi"][0] = 7000.0
    why, n_net, _ = _compare(h2_ar, om_h2_ar, prm, T, p, Y)
    assert why["conservation"] >= 1, why
    assert why["newton"] >= 6, why
    assert n_net >= 20, (why, n_net)
