"""The oracle's pins are sensitive: each ORACLE_MUTANT_* macro plants one
plausible mistake in a separate build of the oracle (on the CPU), and at
least one pin of tests/test_oracle_pins.py must fail against it."""
import os
import tempfile

import pytest

import oracle
from oracle import build as obuild
import test_oracle_pins as pins

PIN_CALLS = [
    ("matern_closed_forms", lambda: [pins.test_matern_closed_forms_match_bessel(nu) for nu in (0.5, 1.5, 2.5)]),
    ("rbf_limit", pins.test_rbf_is_the_matern_limit),
    ("knn_ties", lambda: [pins.test_knn_matches_allpairs_sort_on_tie_heavy_grid(d) for d in (1, 2, 3)]),
    ("blocks", lambda: pins.test_blocks_symmetric_spd_nugget_on_diagonal("matern", 1.5)),
    ("dense_gp", lambda: pins.test_k_equals_n_is_the_dense_gp_mean("matern", 1.5)),
    ("interpolation", pins.test_interpolation_identity),
    ("loo_identity", pins.test_loo_identity_links_loocv_to_precompute),
    ("sigma2", pins.test_sigma2_invariance),
    ("mcmc_posterior", lambda: [pins.test_mcmc_reproduces_the_closed_form_posterior(f) for f in (1.5, 0.15)]),
    ("mcmc_greedy", pins.test_mcmc_takes_only_strictly_better_moves_when_expo_is_zero),
]

MUTANTS = {
    "ORACLE_MUTANT_RBF_SCALE": "RBF read as exp(-d^2/rho^2)",
    "ORACLE_MUTANT_MATERN_POLY": "Matern 3/2 polynomial without sqrt(3)",
    "ORACLE_MUTANT_NUGGET_UNSCALED": "nugget added without sigma^2",
    "ORACLE_MUTANT_SELF_LAST": "S_i with the point itself last",
    "ORACLE_MUTANT_CROSS_NUGGET": "nugget in the cross-covariance",
    "ORACLE_MUTANT_LOO_SIGN": "LOO residual sign flipped",
    "ORACLE_MUTANT_BACKSOLVE_TRANSPOSE": "back substitution with L instead of L^T",
    "ORACLE_MUTANT_TIE_HIGH": "distance ties to the highest index",
    "ORACLE_MUTANT_MCMC_SIGN": "Metropolis log ratio with the sign flipped",
    "ORACLE_MUTANT_MCMC_NO_HALF": "Gaussian log likelihood without the 1/2",
}


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory() as d:
        yield d


def _failing_pins():
    failed = []
    for name, call in PIN_CALLS:
        try:
            call()
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(name)
    return failed


def test_pins_pass_on_the_real_oracle():
    assert _failing_pins() == []


@pytest.mark.parametrize("macro", sorted(MUTANTS))
def test_a_planted_mistake_fails_a_pin(workdir, macro):
    path = obuild.build_variant([macro], os.path.join(workdir, f"lib_{macro}.so"))
    with oracle.use_library(path):
        failed = _failing_pins()
    assert failed, f"no pin caught: {MUTANTS[macro]}"
