"""Why the network stays FP32: the per-species network of Sec. "model" evaluated on the
oracle's descriptors of the bench model, with its inputs q~ and weights W0 rounded as a
tensor-core GEMM would take them (TF32: 10 mantissa bits, BF16: 7; products exact, sums
kept in higher precision, so the errors below are lower bounds), against FP64.

On 40 FCC/BCC structures BF16 misses the mixed-precision energy bound (0.1 meV/atom on
|Delta E_s| / N_a) by an order of magnitude, and TF32 reaches it.  Inputs rounded to FP32
stay three orders of magnitude inside it."""
import numpy as np

import oracle
from paper_2606_19557_gb300 import synth


def _round_mantissa(x, bits):
    """float32 values rounded to nearest (ties to even) at `bits` explicit mantissa bits."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    if bits >= 23:
        return np.asarray(x, np.float32).astype(np.float64)
    drop = np.uint64(23 - bits)
    lsb = (u >> drop) & np.uint64(1)
    u = ((u + (np.uint64(1) << (drop - np.uint64(1))) - np.uint64(1) + lsb) >> drop) << drop
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _energies(spec, theta, qt, types, bits):
    T, NN, ND = spec.n_types, spec.n_neu, qt.shape[1]
    w0 = theta[:T * NN * ND].reshape(T, NN, ND)
    o = T * NN * ND
    b0 = theta[o:o + T * NN].reshape(T, NN)
    o += T * NN
    w1 = theta[o:o + T * NN].reshape(T, NN)
    b1 = theta[o + T * NN]
    E = np.zeros(len(qt))
    for t in range(T):
        m = types == t
        A, W = qt[m], w0[t]
        if bits is not None:
            A, W = _round_mantissa(A, bits), _round_mantissa(W, bits)
        E[m] = np.tanh(A @ W.T - b0[t]) @ w1[t] - b1
    return E


def test_rounding_mantissa():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -9, -3.0 - 2.0 ** -7], np.float32)
    np.testing.assert_array_equal(_round_mantissa(x, 7), [1.0, 1.0, 1.0 + 2.0 ** -7, 1.0, -3.0])


def test_network_precision_against_energy_bound():
    spec = synth.SPECS["fcc_bcc_t1"]
    b = synth.batch_fcc_bcc(seed=2, n_struct=40)
    theta = synth.random_theta(oracle.num_params(spec), 1)
    q = oracle.descriptors(spec, theta, b)
    qt = q * oracle.scale_from_range(q).astype(np.float32).astype(np.float64)
    types = np.asarray(b.types)
    off = np.asarray(b.atom_off)
    E64 = _energies(spec, theta, qt, types, None)

    def per_structure_mev(bits):
        dE = _energies(spec, theta, qt, types, bits) - E64
        return np.abs(np.add.reduceat(dE, off[:-1]) / np.diff(off)) * 1e3

    fp32, tf32, bf16 = per_structure_mev(23), per_structure_mev(10), per_structure_mev(7)
    assert fp32.max() < 1e-3
    assert bf16.max() > 1.0 and np.median(bf16) > 0.5  # 10x the 0.1 meV/atom bound
    assert tf32.max() > 0.1                            # at the bound
