"""CPU checks of the kernel-source hash behind bench.py's `traffic` field: it
ignores comments and blank space but not code."""
from paper_2203_15561_gb300 import kernel_hash as kh


def test_code_only_ignores_comments_and_blank_space():
    a = "int f(int x) {\n  return x + 1;  // add one\n}\n/* block\n comment */\n"
    b = "int  f(int x){return x+1;}"
    assert kh._code_only(a) == kh._code_only(b)
    assert kh._code_only(a) != kh._code_only(a.replace("x + 1", "x + 2"))


def test_source_hash_is_stable_and_short():
    h = kh.source_hash()
    assert h == kh.source_hash() and len(h) == 16 and int(h, 16) >= 0


def test_source_hash_follows_code_not_comments(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k(int* p) { *p = 1; }  // one\n")
    h0 = kh.source_hash([src])
    src.write_text("// a new comment\n__global__ void k(int* p) {\n  *p = 1;\n}\n")
    assert kh.source_hash([src]) == h0
    src.write_text("__global__ void k(int* p) { *p = 2; }\n")
    assert kh.source_hash([src]) != h0
