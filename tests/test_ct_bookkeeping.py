"""Host bookkeeping of the combination technique (Section IV-B) in the package against the
oracle's index sets, plus identities of the sets themselves.  No GPU work runs here."""
import pytest

import oracle as O

ct = pytest.importorskip("paper_2308_01457_gb300.ct")


@pytest.mark.parametrize("L0", range(0, 4))
@pytest.mark.parametrize("L", range(0, 8))
def test_index_sets_and_hermitian_blocks_match_the_oracle(L0, L):
    if L < L0:
        pytest.skip("L >= L0")
    plus, minus = ct.index_sets(L0, L)
    assert (plus, minus) == O.ct_index_sets(L0, L)
    assert ct.hermitian_blocks(L0, L) == O.ct_hermitian_blocks(L0, L)
    # the two diagonals l1 + l2 = L + L0 and L + L0 - 1 inside [L0, L]^2
    assert all(a + b == L + L0 and L0 <= a <= L and L0 <= b <= L for a, b in plus)
    assert all(a + b == L + L0 - 1 and L0 <= a <= L and L0 <= b <= L for a, b in minus)
    assert len(plus) == L - L0 + 1 and len(minus) == (L - L0 if L > L0 else 0)
    # the Hermitian reduction covers each set exactly once with its mirror
    herm = ct.hermitian_blocks(L0, L)
    for blocks, sign in ((plus, 1), (minus, -1)):
        mine = [b for b, s in herm if s == sign]
        covered = sorted(set(mine) | {(b, a) for a, b in mine})
        assert covered == sorted(blocks)


def test_dofs_of_the_sphere_levels():
    n = {l: 120 * 4**l for l in range(6)}
    total, biggest = ct.dofs(n, 0, 4)
    plus, minus = ct.index_sets(0, 4)
    assert total == sum(n[a] * n[b] for a, b in plus + minus)
    assert biggest == n[4] * n[0] == n[3] * n[1] == n[2] * n[2]
