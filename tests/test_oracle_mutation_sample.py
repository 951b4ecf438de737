"""A sample of the oracle mutation check (tests/oracle_mutations.py) in the
CPU suite: three planted mistakes, in the energy, the LM damping and the
colour check, must each fail a pin.  The full list runs by hand."""
import shutil

import pytest

from tests import oracle_mutations


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc to build the scratch oracle")
def test_planted_mistakes_fail_a_pin(capsys):
    missed = oracle_mutations.main(["energy squared", "LM Levenberg damping", "colour L1"])
    out = capsys.readouterr().out
    assert out.count("CAUGHT") == 3, out
    assert missed == 0, out
