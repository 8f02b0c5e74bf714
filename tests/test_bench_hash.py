"""The benchmark keys its ncu DRAM-traffic figure by a hash of the operator's kernel sources; edits to
comments or whitespace keep the figure, any code edit drops it (bench.py reports traffic null then).
CPU only."""
import bench


def test_code_only_drops_comments_and_whitespace_but_keeps_strings():
    src = 'int a = 1; // one\n/* block\n comment */ asm("add.rn.f32x2 %0, %1; // not a comment");\n'
    assert bench._code_only(src) == 'int a = 1; asm("add.rn.f32x2 %0, %1; // not a comment");'
    assert bench._code_only(src) == bench._code_only(src.replace("// one", "// two").replace("  ", " "))
    assert bench._code_only(src) != bench._code_only(src.replace("a = 1", "a = 2"))

