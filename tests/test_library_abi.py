"""CPU checks of the C ABI boundary: the library builds, loads, and exports
every function include/genasm.h declares (no GPU calls)."""
import re
import subprocess
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    text = (ROOT / "include" / "genasm.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ga_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2203_15561_gb300 import _build
    so = _build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", str(so)], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(ga_\w+)", out))
    declared = declared_functions()
    assert declared, "no declarations parsed"
    missing = [f for f in declared if f not in exported]
    assert not missing, missing


def test_library_loads_and_reports_version():
    import paper_2203_15561_gb300 as ga
    assert ga.ga_version() >= 100
    assert ga.lib().ga_strerror(ga.GA_EINVAL) == b"invalid argument"


def test_bad_arguments_rejected_before_any_cuda_call():
    import ctypes
    import paper_2203_15561_gb300 as ga
    L = ga.lib()
    sz = ctypes.c_size_t(0)
    assert L.ga_workspace_size(10, 0, 0, 1, ctypes.byref(sz)) == ga.GA_EINVAL
    assert L.ga_workspace_size(10, 64, 64, 1, ctypes.byref(sz)) == ga.GA_EINVAL
    assert L.ga_workspace_size(10, 64, 24, -1, ctypes.byref(sz)) == ga.GA_EINVAL
    assert L.ga_workspace_size(10, 64, 24, 1, None) == ga.GA_EINVAL
    args = [None] * 6 + [5, 64, 24, 64] + [None] * 8
    assert L.ga_align_plain(*args, None) == ga.GA_EINVAL       # NULL buffers, n_pairs > 0
    assert L.ga_align_ablation(*args, 0, None, None, 0, None) == ga.GA_EINVAL
    assert L.ga_align_ablation(*([None] * 6 + [0, 64, 24, 64] + [None] * 8), 4, None, None, 0,
                               None) == ga.GA_EINVAL          # variant outside 0..3
    assert L.ga_ablation_workspace_size(10, 64, 24, 64, 7, ctypes.byref(sz)) == ga.GA_EINVAL
    for bad in (0xE5, 0x1E4, -1, 0):   # not a permutation of the four edge kinds
        assert L.ga_align_batch_order(*([None] * 6 + [0, 64, 24, 64] + [None] * 8), bad, None, 0,
                                      None) == ga.GA_EINVAL
    assert ga.tb_order_code("MSID") == ga.GA_TB_ORDER_DEFAULT
    assert L.ga_pack_2bit(None, 16, None, None, None) == ga.GA_EINVAL
    assert L.ga_measure_int_peak(None, None) == ga.GA_EINVAL
    assert L.ga_measure_smem_peak(None, None) == ga.GA_EINVAL
    assert L.ga_pack_2bit(None, 0, None, None, None) == ga.GA_OK  # nothing to do


def test_oracle_is_not_reachable_from_the_package():
    pkg = ROOT / "paper_2203_15561_gb300"
    for f in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")) + list(pkg.rglob("*.h")):
        text = f.read_text()
        assert "import oracle" not in text and "from oracle" not in text and "genasm_oracle" not in text, f
