"""Gradient comparison by parameter block: the network weights of each species, the shared
output bias and the descriptor coefficients of each ordered species pair differ in size by
orders of magnitude, so one norm over all P entries could hide a wrong block."""
import numpy as np

from paper_2606_19557_gb300 import param_blocks


def block_errors(g, go, spec) -> dict:
    """Relative error ||g_B - go_B|| / ||go_B|| of every block B whose oracle norm is nonzero,
    and for blocks that are zero in the oracle the error relative to the whole gradient."""
    g = np.asarray(g, np.float64).reshape(-1)
    go = np.asarray(go, np.float64).reshape(-1)
    assert g.shape == go.shape
    scale = max(np.linalg.norm(go), 1e-300)
    out = {}
    for name, sl in param_blocks(spec).items():
        nb = np.linalg.norm(go[sl])
        out[name] = float(np.linalg.norm(g[sl] - go[sl]) / (nb if nb > 0 else scale))
    return out


def assert_grad_close(g, go, spec, tol):
    err = block_errors(g, go, spec)
    bad = {k: v for k, v in err.items() if not v <= tol}
    assert not bad, f"blocks above {tol}: {dict(sorted(bad.items(), key=lambda kv: -kv[1])[:8])}"
    return err
