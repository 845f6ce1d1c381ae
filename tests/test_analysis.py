"""Critical-path bound and overlap metrics against brute force.  CPU only."""
import random

import pytest

from oracle import dag as D
from oracle import overlap as O
from paper_2012_09646_gb300 import analysis as A


def test_overlap_worked_example():
    # Section IV-F in miniature: one kernel [0, 10) and one copy [5, 15)
    m = A.overlap_metrics([(0, 10)], [(5, 15)])
    assert m == {"CT": 0.5, "TC": 0.5, "CC": 0.0, "TOT": 0.5}
    # a copy overlapped by two kernels counts once
    m = A.overlap_metrics([(0, 10), (0, 10)], [(0, 10)])
    assert m["TC"] == 1.0 and m["CC"] == 1.0 and m["CT"] == 1.0


@pytest.mark.parametrize("seed", range(30))
def test_overlap_matches_bruteforce(seed):
    rng = random.Random(seed)
    def iv():
        a = rng.randint(0, 60)
        return (a, a + rng.randint(0, 25))
    comp = [iv() for _ in range(rng.randint(0, 6))]
    tran = [iv() for _ in range(rng.randint(0, 6))]
    got = A.overlap_metrics(comp, tran)
    want = O.overlaps_bruteforce(comp, tran)
    for k in want:
        assert got[k] == pytest.approx(want[k], abs=1e-12), k


@pytest.mark.parametrize("seed", range(30))
def test_critical_path_matches_bruteforce(seed):
    rng = random.Random(seed)
    L = rng.randint(1, 12)
    from tests.test_oracle_dag import random_program
    elems = random_program(rng, L, rng.randint(1, 4))
    edges = D.expected_edges(elems)
    w = [rng.uniform(0.1, 5.0) for _ in range(L)]
    assert A.critical_path(w, edges) == pytest.approx(O.longest_path_bruteforce(w, edges))
