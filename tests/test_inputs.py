"""The seeded input generators: SplitMix64 (Steele, Lea and Flood, OOPSLA
2014) against the published output sequences of its reference
implementation, and the uniform draws built on it."""
from paper_1003_4322_gb300 import inputs


def test_splitmix64_matches_the_published_sequences():
    # first outputs of the generator started at state 0 and at state 1234567
    assert [inputs.splitmix64(0, c) for c in (1, 2, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [inputs.splitmix64(1234567, c) for c in (1, 2, 3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_uniform_draws_are_the_top_53_bits():
    for seed, ident, draw in ((0, 0, 0), (7, 12345, 2), (4999, 47, 0)):
        u = inputs.uniform(seed, ident, draw)
        z = inputs.splitmix64(seed, 1 + 3 * ident + draw)
        assert 0.0 <= u < 1.0 and u == (z >> 11) / 2.0 ** 53
