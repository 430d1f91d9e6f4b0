"""The C-ABI library loads, exports every entry point its header declares, and rejects
invalid configurations on the host before touching a GPU.  CPU only."""
import ctypes

import pytest

import paper_2606_19557_gb300 as pkg


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.load_library()


def test_header_lists_the_boundary():
    names = pkg.declared_symbols()
    for n in ("nep_create", "nep_destroy", "nep_set_params", "nep_set_structures", "nep_eval", "nep_loss_grad",
              "nep_backward", "nep_descriptor_range", "nep_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in pkg.declared_symbols() if not hasattr(lib, n)]
    assert missing == []


def _cfg(**kw):
    base = dict(n_types=1, rc_R=5.0, rc_A=4.0, n_max_R=4, n_max_A=4, basis_R=8, basis_A=8, l_max=4, has_4b=0,
                has_5b=0, n_neuron=10, precision=0, device=0)
    base.update(kw)
    return pkg._Config(**base)


@pytest.mark.parametrize("bad", [dict(n_types=0), dict(n_types=17), dict(rc_A=6.0), dict(rc_R=-1.0),
                                 dict(l_max=5), dict(has_4b=1, l_max=1), dict(n_neuron=0), dict(n_neuron=129),
                                 dict(n_max_R=12), dict(basis_A=12), dict(precision=7)])
def test_invalid_config_rejected_on_host(lib, bad):
    h = ctypes.c_void_p()
    rc = lib.nep_create(ctypes.byref(_cfg(**bad)), None, ctypes.byref(h))
    assert rc == pkg.NEP_EINVAL
    assert h.value is None
    assert len(lib.nep_last_error(None)) > 0


def test_null_handles_rejected(lib):
    P = ctypes.c_int64()
    assert lib.nep_num_params(None, ctypes.byref(P)) == pkg.NEP_EINVAL
    assert lib.nep_eval(None, None, None, None) == pkg.NEP_EINVAL
    assert lib.nep_loss_grad(None, None, None, None, None, 1.0, 1.0, 1.0, None, None) == pkg.NEP_EINVAL
    lib.nep_destroy(None)


def test_param_blocks_partition_theta():
    """The parameter blocks the gradient checks use cover theta [0, P) exactly, in the
    header's order, and put b1 where the oracle's hand-worked loss fixture has its only
    nonzero derivative."""
    import oracle
    from paper_2606_19557_gb300 import synth
    for name, spec in synth.SPECS.items():
        blocks = list(pkg.param_blocks(spec).values())
        assert blocks[0].start == 0 and blocks[-1].stop == oracle.num_params(spec), name
        assert all(a.stop == b.start and a.stop > a.start for a, b in zip(blocks, blocks[1:])), name
    spec = synth.SPECS["fcc_bcc_t1"]
    b1 = pkg.param_blocks(spec)["b1"]
    nd = oracle.num_descriptors(spec)
    assert b1.start == spec.n_types * (nd + 2) * spec.n_neu and b1.stop == b1.start + 1
