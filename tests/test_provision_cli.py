"""The provisioning command line's configuration arguments (host logic): Table 4's levels, the fixed configuration
PP-STAT uses and further named (degree, Pre-BTS, Newton steps) configurations such as the paper's own HE-DAP
choice (254, 0, 4) at level 12 (Table 4)."""
import pytest

from paper_2606_10477_gb300 import provision


def test_named_configurations_parse():
    assert provision.parse_configs("254,0,4;126,0,5;126,1,4") == [(254, 0, 4), (126, 0, 5), (126, 1, 4)]
    assert provision.parse_configs("") == []
    assert provision.parse_configs("62,0,7;") == [(62, 0, 7)]
    assert provision.parse_fixed("510,6") == (510, 6)
    assert provision.parse_levels("12,7") == [12, 7]
    assert provision.parse_levels("") == []


@pytest.mark.parametrize("bad", ["254,2,4", "254,0", "0,0,4", "254,0,-1", "a,b,c"])
def test_malformed_configurations_are_refused(bad):
    with pytest.raises(ValueError):
        provision.parse_configs(bad)


@pytest.mark.parametrize("bad", ["510", "510,6,1", "0,6", "510,-1"])
def test_malformed_fixed_configuration_is_refused(bad):
    with pytest.raises(ValueError):
        provision.parse_fixed(bad)
