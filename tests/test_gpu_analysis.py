"""The analysis tail driven by the library: logarithmic bins run on the GPU."""
import numpy as np
import pytest

import hsg_inputs as gi
from paper_1309_1599_b300 import analysis as an
from _gpu_helpers import make

pytestmark = pytest.mark.gpu


def test_log_binned_run_equals_the_explicit_bin_sequence():
    """run_log_binned gives bins of base, base, 2 base, 4 base, ... steps:
    the same means as resetting and running those lengths by hand on an
    identical lattice."""
    betas = gi.linear_betas(0.3, 1.0, 4)
    a, _ = make([8, 8, 8], betas, n_rep=2, n_or=2, measure_every=1)
    b, _ = make([8, 8, 8], betas, n_rep=2, n_or=2, measure_every=1)
    bins = an.run_log_binned(a, n_bins=5, base_steps=2)
    assert bins.shape == (5, 3, 4, 9)
    for i, n in enumerate([2, 2, 4, 8, 16]):
        b.reset_observables()
        b.run_steps(n)
        obs, counts = b.read_observables()
        assert np.all(counts == n)
        assert np.array_equal(bins[i], an.observable_means(obs, counts, 2))
    delta, err = an.thermalization_test(np.transpose(bins, (1, 0, 2, 3)))
    assert delta.shape == (5, 4, 9) and np.all(delta[-1] == 0)
    chi = an.susceptibilities(bins[-1], 8 ** 3)
    xi = an.xi_second_moment(chi["sg0"], chi["sgk"], 8)
    assert xi.shape == (3, 4)
    with pytest.raises(ValueError):
        c, _ = make([8], betas, n_rep=2, measure_every=3)
        an.run_log_binned(c, n_bins=2, base_steps=2)
