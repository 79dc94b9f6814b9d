"""The pins catch plausible mistakes: each ORC_PLANT variant of the oracles (a
dropped term, a wrong sign, weight, factor or index, a transposed matrix, a
missing clip) must fail the oracle's pin suite, while the unplanted oracle
passes it (the rest of this directory)."""
import os
import subprocess
import sys

import pytest

from conftest import ROOT

PLANTS = {
    1: "u.grad(rho) dropped from the forcing term (Eq. 21)",
    2: "sign of the y-gradient stencil flipped (Sec. 3.2)",
    3: "weight of g_eq at i = 0 wrong (Eq. 31)",
    4: "transposed M in the collision (Eqs. 24-25)",
    5: "F instead of F/2 in the velocity (Eq. 28)",
    6: "d_t(phi u) dropped from the source (Eq. 32)",
    7: "kappa doubled (Sec. 2)",
    8: "no clip of phi before psi (Eq. 37)",
    9: "rho s_0(u) dropped from the pressure (Eq. 29)",
    10: "sign of the sharpening flux flipped (Eq. 32)",
    21: "sign of the moving-wall momentum term flipped (halfway bounce-back)",
    22: "periodic ghost row at the walls instead of the mirrored one",
    24: "cos(2 pi t/T) for the time factor of the single vortex (Eqs. 43-44)",
    25: "X and Y swapped in the single vortex (Eqs. 43-44)",
    26: "single-vortex coordinates x/L without the half-node offset (Eqs. 43-44)",
    27: "sin instead of sin^2 in the single vortex's u (Eq. 43)",
}
PIN_FILES = ["tests/test_oracle_lattice.py", "tests/test_oracle_node.py",
             "tests/test_oracle_stencil.py", "tests/test_oracle_physics.py",
             "tests/test_oracle_walls.py", "tests/test_oracle_vortex.py"]


@pytest.mark.parametrize("plant", sorted(PLANTS), ids=lambda k: f"plant{k}")
def test_planted_mistake_is_caught(plant):
    import oracle
    oracle.build(plant=plant)
    env = dict(os.environ, ORACLE_PLANT=str(plant))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *PIN_FILES], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"pins did not catch: {PLANTS[plant]}\n{r.stdout[-2000:]}"


PLANTS3 = {
    11: "-c_s^2 I dropped from the forcing tensor (Eq. 21, D3Q19)",
    12: "D3Q19 sound speed used in the D3Q7 g_eq (Eq. 31)",
    13: "sign of the z-gradient stencil flipped (Sec. 3.2, D3Q19)",
    14: "F instead of F/2 in the velocity (Eq. 28)",
    15: "d_t(phi u) dropped from the source (Eq. 32)",
    16: "sign of the sharpening flux flipped (Eq. 32)",
    17: "D2Q9 weight w_0 in the pressure prefactor (Eq. 29)",
    18: "wrong face-diagonal weight in the stencils (Sec. 3.2)",
    19: "g streamed against c_z",
    20: "tau_f from mu(phi)/rho_l instead of mu(phi)/rho(phi) (Eq. 27)",
    23: "unit normal of Eq. 17 down to |grad psi| = 0 (no ridge cut)",
}


@pytest.mark.parametrize("plant", sorted(PLANTS3), ids=lambda k: f"plant{k}")
def test_planted_mistake_is_caught_3d(plant):
    import oracle
    oracle.build3(plant=plant)
    env = dict(os.environ, ORACLE_PLANT=str(plant))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not slow", "tests/test_oracle3d.py"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch: {PLANTS3[plant]}\n{r.stdout[-2000:]}"
