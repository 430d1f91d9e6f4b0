"""Gradient comparison by parameter block: the network weights of each species, the shared
output bias and the descriptor coefficients of each ordered species pair differ in size by
orders of magnitude, so one norm over all P entries could hide a wrong block.

A block B passes when its error is within `tol` of its own oracle norm, or, for a block
whose value is a near-cancelling sum (FP32 rounding of the terms then exceeds tol of the
small result), within tol/10 of the whole gradient's norm.  A block off by 1e-2 of itself
therefore fails unless it is below 1e-4 of the gradient, where it cannot matter."""
import numpy as np

from paper_2606_19557_gb300 import param_blocks


def block_errors(g, go, spec) -> dict:
    """(relative error of block B, its error relative to the whole gradient) per block."""
    g = np.asarray(g, np.float64).reshape(-1)
    go = np.asarray(go, np.float64).reshape(-1)
    assert g.shape == go.shape
    scale = max(np.linalg.norm(go), 1e-300)
    out = {}
    for name, sl in param_blocks(spec).items():
        nb = np.linalg.norm(go[sl])
        err = np.linalg.norm(g[sl] - go[sl])
        out[name] = (float(err / nb) if nb > 0 else float("inf") if err > 0 else 0.0, float(err / scale))
    return out


def assert_grad_close(g, go, spec, tol):
    err = block_errors(g, go, spec)
    bad = {k: v for k, v in err.items() if not (v[0] <= tol or v[1] <= 0.1 * tol)}
    assert not bad, f"blocks above {tol}: {dict(sorted(bad.items(), key=lambda kv: -kv[1][0])[:8])}"
    return err
