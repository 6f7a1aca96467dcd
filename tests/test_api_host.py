"""Host-side argument checks of the Python binding that need no GPU."""
import pytest


def test_dslash_rejects_bad_parity():
    import paper_1801_01473_gb300 as p
    with pytest.raises(ValueError):
        p.dslash(None, 2, None)
