"""The package's smoke check (one small step on cuda:0 against the oracle)
runs as part of the GPU suite, so that a change that breaks it is caught."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point(gs):
    import __graft_entry__

    __graft_entry__.smoke()
