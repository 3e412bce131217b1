"""CPU checks of the ncu summary tool behind profiles/ and bench.py's
`traffic` field: the kernel-source hash ignores comments and blank space but
not code, and the launch table sums times and shares per kernel."""
from paper_2203_15561_gb300 import ncu_summary as ns


def test_code_only_ignores_comments_and_blank_space():
    a = "int f(int x) {\n  return x + 1;  // add one\n}\n/* block\n comment */\n"
    b = "int  f(int x){return x+1;}"
    assert ns._code_only(a) == ns._code_only(b)
    assert ns._code_only(a) != ns._code_only(a.replace("x + 1", "x + 2"))


def test_source_hash_is_stable_and_short():
    h = ns.source_hash()
    assert h == ns.source_hash() and len(h) == 16 and int(h, 16) >= 0


def test_launch_table_sums_per_kernel(tmp_path):
    csv = tmp_path / "launches.csv"
    rows = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    data = [("0", "void ga::a_kernel<8>(int)", "msecond", "2"),
            ("1", "ga::b_kernel(int)", "usecond", "500"),
            ("2", "void ga::a_kernel<8>(int)", "nsecond", "1,000,000"),
            ("3", "ga::c_kernel(int)", "msecond", "7")]
    for i, k, u, v in data:
        rows.append(f'"{i}","{k}","gpu__time_duration.sum","{u}","{v}"')
    csv.write_text("==PROF== preamble\n" + "\n".join(rows) + "\n")
    table = ns.launches(str(csv), 0, 3).splitlines()
    assert table[2] == "| `ga::a_kernel<8>` | 2 | 3.000 | 85.7% |"
    assert table[3] == "| `ga::b_kernel` | 1 | 0.500 | 14.3% |"
    assert len(table) == 4  # the fourth launch is outside the slice
