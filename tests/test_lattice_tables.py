"""The product's 37-velocity table (generated header) against its generator and
against the oracle's independent derivation of the same quadrature."""
from paper_1808_04406_gb300 import gen_d2q37


def test_committed_header_is_the_generator_output():
    with open(gen_d2q37.HEADER) as fh:
        assert fh.read() == gen_d2q37.header_text()


def test_generator_and_oracle_derive_the_same_rule():
    """Two different 50-digit solves (determinant root + least squares in the
    oracle; x^8-residual root + 8 x 8 solve in the generator) round to the same
    FP64 scale and weights."""
    import oracle
    import oracle.h37 as H
    oracle.lib()
    e, w, c = gen_d2q37.solve()
    eo, wo, co = H.lattice()
    assert c == co
    ref = {tuple(v): x for v, x in zip(eo, wo)}
    assert sorted(ref) == sorted(tuple(v) for v in e)
    assert all(ref[tuple(v)] == x for v, x in zip(e, w))
    assert all((e[i] == -e[36 - i]).all() for i in range(37))


def test_rule_generator_matches_the_oracle_rules():
    """The library's rule generator (exact-cofactor polynomial in 1/c^2) and the
    oracle's (determinant scan and bisection, normal equations) find the same
    eight minimal rules, bit for bit in FP64."""
    from oracle import hlat
    from paper_1808_04406_gb300 import gen_rules
    for degree in (7, 9):
        mine, theirs = gen_rules.rules(degree), hlat.rule_set(degree)
        assert [r[0] for r in mine] == [r[0] for r in theirs] == ["A", "B", "C", "D"]
        for (_, e, w, c), (_, eo, wo, co) in zip(mine, theirs):
            assert c == co
            lut = {tuple(v): x for v, x in zip(eo, wo)}
            assert len(e) == len(eo) and all(lut[tuple(v)] == x for v, x in zip(e, w))
