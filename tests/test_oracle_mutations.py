"""The oracle's pins must catch plausible mistakes.

Each case compiles the oracle with one deliberate mistake (a PLANT_* switch of
``oracle/bd_oracle.c``; CPU only) and runs the pins of
``test_oracle_pins.py`` against that build.  At least one pin has to fail.
"""
import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

PINS = [
    pins.test_alpha_independence,
    pins.test_translation_invariance,
    lambda: pins.test_hasimoto_self_mobility(7.7),
    lambda: pins.test_free_space_rpy_recovery(0.6),
    lambda: pins.test_free_space_rpy_recovery(2.5),
    pins.test_symmetry_and_positive_definite,
    pins.test_mstar_C1_continuity_at_2a,
    pins.test_coincident_limit_equals_self_block,
    pins.test_divergence_free,
    pins.test_forces_hookean_fene_closed_form,
    pins.test_cheb_scalar_matrix,
    pins.test_cheb_converges_to_eigen_root_and_SS_equals_D,
    pins.test_step_closed_form_with_identity_D,
]

PLANTS = {
    "PLANT_PRINTED_MSTAR": "rr coefficient of M* as printed in Eq. (cor5)",
    "PLANT_RECIP_SIGN": "minus sign of the reciprocal bracket of Eq. (DF) as printed",
    "PLANT_SELF_SIGN": "sign of the alpha^3 self term flipped",
    "PLANT_M1_COEF": "one coefficient of Eq. (M1) changed (20 -> 16)",
    "PLANT_M2_VOLUME": "1/V in Eq. (M2) replaced by 1/L^2",
    "PLANT_CHEB_NO_HALF": "the -c_0/2 dW term of Eq. (cheb1) dropped",
    "PLANT_CHEB_RECURRENCE": "sign of V_{p-2} in Eq. (cheb2) flipped",
    "PLANT_STEP_DRIFT": "dt/4 of Eq. (sde) replaced by dt/2",
    "PLANT_SPRING_SIGN": "reaction force of a spring given the wrong sign",
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_pins_catch_planted_mistake(plant):
    failed = []
    with oracle.variant(plant):
        for f in PINS:
            try:
                f()
            except (AssertionError, np.linalg.LinAlgError):
                failed.append(getattr(f, "__name__", "lambda"))
    assert failed, f"no pin caught: {PLANTS[plant]}"
