"""C-ABI library checks that need no GPU: it loads, exports every declared
symbol, and its host-side configuration tables agree with the oracle."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(gs_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    import paper_2607_06604_gb300 as gs
    lib = ctypes.CDLL(gs.lib_path)
    names = declared_symbols()
    assert len(names) >= 12, names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_num_configs_match_oracle():
    import paper_2607_06604_gb300 as gs
    for nb in (1, 2, 5, 10, 15, 20, 254):
        assert gs.gs_num_configs(3, nb) == oracle.num_configs(3, nb)
    for nb in range(1, 9):
        assert gs.gs_num_configs(4, nb) == oracle.num_configs(4, nb)


@pytest.mark.parametrize("nb", [1, 2, 3, 4, 6])
def test_config_tables_match_oracle(nb):
    import paper_2607_06604_gb300 as gs
    for k in range(gs.gs_num_configs(4, nb)):
        assert gs.gs_config_bins(4, nb, k) == oracle.config_bins(4, nb, k)
    for k in range(gs.gs_num_configs(3, nb + 6)):
        assert gs.gs_config_bins(3, nb + 6, k) == oracle.config_bins(3, nb + 6, k)


def test_host_argument_errors():
    import paper_2607_06604_gb300 as gs
    with pytest.raises(gs.GSError) as e:
        gs.gs_num_configs(5, 4)
    assert e.value.status == -1
    with pytest.raises(gs.GSError) as e:
        gs.gs_num_configs(4, 17)
    assert e.value.status == -2
    with pytest.raises(gs.GSError) as e:
        gs.gs_config_bins(3, 4, 20)
    assert e.value.status == -2
    xyz = np.zeros((4, 3), np.int32)
    # edges not strictly increasing, rmax >= L/4, too many bins: rejected on the host
    for edges, box in (([0, 10, 10], 1000), ([0, 300], 1000), (list(range(300)), 10 ** 6)):
        with pytest.raises(gs.GSError) as e:
            gs.gs_build_graph(xyz, box, edges)
        assert e.value.status == -2
    assert gs.gs_strerror(-5) == "bounded device wait expired"
