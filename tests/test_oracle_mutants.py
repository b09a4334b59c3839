"""Planted mistakes in the FP64 oracle are caught by its pins.

Each case edits one oracle function's source text in one place (a dropped
conjugate, a transposed weight, a flipped tap, ...), compiles the edited
function in the oracle's own namespace, patches it into the module for the
duration of the test, and runs the pin that should catch that kind of
mistake: the pin must fail.  This keeps the claim "a plausible mistake
anywhere in the oracle fails a pin" checkable on CPU.
"""
import inspect

import pytest

from oracle import nrx_oracle as O
from tests import test_oracle_pins as P

# (name, oracle function, text, replacement, pin, pin arguments)
MUTANTS = [
    ("dropped conjugate in LS", "ls_estimates", "np.conj(p)[None, :]", "p[None, :]",
     P.test_ls_exact_on_noiseless_pilots_single_port, (1,)),
    ("OCC estimate position", "ls_estimates", "pos = 4.0 * np.arange(M // 2) + 1.0 + g",
     "pos = 4.0 * np.arange(M // 2) + g", P.test_ls_exact_with_occ_when_flat_over_pilot_pair, ()),
    ("time interpolation weight", "interpolate", "a = (t - t0) / (t1 - t0)", "a = (t1 - t) / (t1 - t0)",
     P.test_interpolation_exact_on_affine_channel, (1, (2, 11))),
    ("PE sign", "positional_encoding", "((s - nearest_s) / 2.0)", "((nearest_s - s) / 2.0)",
     P.test_positional_encoding_hand_values, ()),
    ("transposed weight", "dense", "np.asarray(w, dtype=np.float64).T", "np.asarray(w, dtype=np.float64)",
     P.test_dense_matches_torch_linear, ()),
    ("flipped depthwise tap", "depthwise3x3", "k[:, i, j]", "k[:, 2 - i, 2 - j]",
     P.test_depthwise_matches_scipy_and_torch, ()),
    ("missing ReLU", "relu", "np.maximum(x, 0.0)", "x", P.test_nrx_forward_matches_torch_layer_stack, (2,)),
    ("self-message in aggregation", "aggregate", "if v != u:", "if True:",
     P.test_single_user_aggregate_is_zero_and_inactive_users_ignored, ()),
    ("missing residual", "residual_block", "return z + dense(", "return dense(",
     P.test_nrx_forward_matches_torch_layer_stack, (1,)),
    ("swapped CNN input order", "cnn_update", "[S_u, a_u, pe_u]", "[a_u, S_u, pe_u]",
     P.test_nrx_forward_matches_torch_layer_stack, (2,)),
    ("LLR sign", "maxlog_llr", "out[..., i] = d0 - d1", "out[..., i] = d1 - d0",
     P.test_maxlog_qpsk_closed_form, ()),
    ("post-equalisation variance", "lmmse_equalize", "var = 1.0 / d - 1.0", "var = 1.0 / d",
     P.test_lmmse_single_user_is_mrc, ()),
    ("missing conjugate in back substitution", "cholesky_solve", "np.conj(L[..., j, i])", "L[..., j, i]",
     P.test_cholesky_solve_matches_numpy_solve, ()),
]


def _mutant(func_name: str, old: str, new: str):
    src = inspect.getsource(getattr(O, func_name))
    assert src.count(old) == 1, f"the text to mutate must occur once in {func_name}"
    ns = {}
    exec(compile(src.replace(old, new), f"<mutant of {func_name}>", "exec"), O.__dict__, ns)
    return ns[func_name]


@pytest.mark.parametrize("case", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pin(case, monkeypatch):
    name, func_name, old, new, pin, args = case
    pin(*args)  # the pin passes on the oracle as it stands
    monkeypatch.setattr(O, func_name, _mutant(func_name, old, new))
    with pytest.raises(Exception):
        pin(*args)
