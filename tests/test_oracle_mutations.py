"""The oracle's pins catch plausible mistakes planted in the oracle.

Each mutation is compiled into a separate copy of the C oracle
(-DORC_MUTATION=n); nothing here touches the GPU path.  For every mutation at
least one of the distribution pins (test_oracle_law.py) or the Philox pin
(test_oracle_philox.py) must fail.

  1  +g dropped from the acceptance numerator (Eq. 7)
  2  c_k terms of Eq. 7 swapped between source and proposal
  3  wrong mixture weight L / (L + 2G) (Sec. 4.3 footnote)
  4  word proposals drawn from the pre-acceptance assignments
  5  Dice(n) off by one (never returns n - 1)
  7  the document count c_d leaves out the document's last token
  8  every MH step starts from the phase-start z instead of the current state
  9  Philox with 9 rounds instead of 10
 10  fold-in: the frozen word's j-th smallest topic off by one rank
 11  fold-in: pi^doc and the word proposal read a neighbouring token's word row
 12  fold-in: theta normalised by L_d + alpha instead of L_d + alpha_bar
 13  learned fold-in: q(s) and q(t) swapped in the independence-sampler rate
"""
import pytest

import oracle
from tests import test_oracle_law as law
from tests import test_oracle_philox as ph


def _fails(fn):
    try:
        fn()
    except AssertionError:
        return True
    return False


def _law_pins(m):
    checks = []
    for M in (1, 2):
        def doc(M=M):
            oz, op, ex = law.run_doc_law(M, mutation=m)
            law._check_joint(oz, op, tag="doc", **ex)

        def word(M=M):
            oz, op, ex = law.run_word_law(M, mutation=m)
            law._check_joint(oz, op, tag="word", **ex)
        checks += [doc, word]
    return checks


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7, 8])
def test_law_pins_catch_mutation(m):
    assert any(_fails(c) for c in _law_pins(m)), f"mutation {m} not caught"


def test_philox_pin_catches_round_count():
    pytest.importorskip("triton")
    cases = [(42, [[1, 2, 3, 4], [0, 0, 0, 0]])]
    want = ph._triton_philox(cases)[0]
    got = [oracle.philox(c, [42, 0], mutation=9).tolist() for c in cases[0][1]]
    assert got != want
    good = [oracle.philox(c, [42, 0]).tolist() for c in cases[0][1]]
    assert good == want


def test_unmutated_oracle_passes_same_pins():
    assert not any(_fails(c) for c in _law_pins(0))


def _foldin_pins(m):
    from tests import test_oracle_foldin as fo
    return [lambda: fo.check_frozen_word_law(mutation=m),
            lambda: fo.check_theta_rows_normalised(mutation=m),
            lambda: fo.check_separable_words(mutation=m),
            lambda: fo.check_against_cgs(mutation=m)]


@pytest.mark.parametrize("m", [10, 11, 12])
def test_foldin_pins_catch_mutation(m):
    assert any(_fails(c) for c in _foldin_pins(m)), f"mutation {m} not caught"


def test_learned_pin_catches_mutation():
    from tests import test_oracle_learned as le
    assert _fails(lambda: le.check_learned_against_cgs(mutation=13))
