"""CPU checks of the bench's byte model: every streaming kernel of the time
step that the library's per-kernel timing names has algorithmic bytes, so the
roofline can be taken on whichever kernel dominates."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# named launches that are not fine-grid streaming passes of the forward step:
# latency-bound or plane-sized work, the learned guess and the adjoint
NOT_STREAMING = {"coarsest", "coarsest_fin", "weak_rows", "coarse_operator", "blend_band", "band_copy", "padd", "exit", "tguess_apply", "guess_net", "guess_apply", "force_dparam", "flux_raw"}


def _named_launches():
    src = open(os.path.join(ROOT, "paper_2407_16032_b300", "csrc", "wl_sim.cuh")).read()
    names = set()
    for args in re.findall(r'\b(?:B|P0)\(([^;]*);', src):   # every quoted name in the call's arguments
        names |= set(re.findall(r'"([a-z_0-9]+)"', args))
    flux = re.search(r'names\[7\] = \{([^}]*)\}', src).group(1)
    names |= set(re.findall(r'"([a-z_0-9]+)"', flux))
    return {n for n in names if not n.startswith("adj_")}


def test_every_streaming_kernel_of_the_step_has_algorithmic_bytes():
    names = _named_launches()
    assert {"pcg_dq", "resid", "flux_pred", "grad", "div"} <= names
    missing = [n for n in sorted(names - NOT_STREAMING) if bench.algo_bytes(n, 4, 3) is None]
    assert not missing, missing


def test_byte_model_follows_the_constant_diagonal():
    # a body-free all-periodic grid has one Jacobi diagonal and reads no 1/D
    assert bench.algo_bytes("pcg_u", 4, 3) - bench.algo_bytes("pcg_u", 4, 3, const_diag=True) == 4
    assert bench.algo_bytes("pcg_init", 4, 3) - bench.algo_bytes("pcg_init", 4, 3, const_diag=True) == 4
    assert bench.algo_bytes("pcg_dq", 4, 3) == 16 and bench.algo_bytes("resid", 4, 3) == 4 * (4 + 1 + 1 / 8)
