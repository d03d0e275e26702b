"""Host-side input generation: the seeded ensemble draw (CPU)."""
from paper_1509_02615_gb300 import inputs as inp


def test_ensemble_draw_skips_unstable_pairs_and_is_seeded():
    a = inp.ensemble_members(96, seed=0, spacings=(400.0,))
    b = inp.ensemble_members(96, seed=0, spacings=(400.0,))
    keys = [(m.nodes.layout, m.n, m.l) for m in a]
    assert keys == [(m.nodes.layout, m.n, m.l) for m in b]
    assert not set(keys) & set(inp.ENSEMBLE_UNSTABLE)
    # every stable pair of every layout still occurs
    want = {(lay,) + s for lay in ("cart", "hex", "scattered") for s in inp.ENSEMBLE_STENCILS} - set(inp.ENSEMBLE_UNSTABLE)
    assert set(keys) == want


def test_members_carry_their_hyperviscosity_constant():
    a = inp.ensemble_members(96, seed=0, spacings=(400.0,))
    for m in a:
        want = inp.ENSEMBLE_GAMMA_C.get((m.nodes.layout, m.n, m.l), inp.ENSEMBLE_DEFAULT_GAMMA_C)
        assert m.gamma_c == want
    assert any(m.gamma_c == 2.0 ** -5 for m in a) and any(m.gamma_c == 2.0 ** -6 for m in a)
