"""The benchmark keys its ncu capture records by the CUDA sources' code: a change of
comments or blank lines keeps the key, any change of code (string literals included)
moves it, so traffic figures are reported only for the kernels they were measured on."""

import bench


def _tree(tmp_path, files):
    d = tmp_path / "paper_1006_0532_gb300" / "csrc"
    d.mkdir(parents=True)
    for name, text in files.items():
        (d / name).write_text(text)
    return str(tmp_path)


def _hash_of(root):
    old = bench.ROOT
    try:
        bench.ROOT = root
        return bench.kernel_sources_hash()
    finally:
        bench.ROOT = old


SRC = ('#include "x.h"  // the header\n'
       '/* a block\n   comment */\n'
       '__global__ void k(int* p) {\n'
       '  const char* s = "a // not a comment";\n'
       '  p[0] = \'/\';  // trailing\n'
       '}\n')


def test_comments_and_blank_lines_keep_the_hash(tmp_path):
    a = _hash_of(_tree(tmp_path / "a", {"k.cu": SRC, "x.h": "int f();\n"}))
    reworded = SRC.replace("// the header", "// another remark").replace("a block", "other words")
    b = _hash_of(_tree(tmp_path / "b", {"k.cu": "\n// new note\n" + reworded + "\n\n",
                                        "x.h": "// declared here\nint f();   \n"}))
    assert a == b


def test_code_changes_move_the_hash(tmp_path):
    a = _hash_of(_tree(tmp_path / "a", {"k.cu": SRC}))
    b = _hash_of(_tree(tmp_path / "b", {"k.cu": SRC.replace("p[0]", "p[1]")}))
    c = _hash_of(_tree(tmp_path / "c", {"k.cu": SRC.replace("not a comment", "not a remark")}))
    d = _hash_of(_tree(tmp_path / "d", {"k.cu": SRC, "new.cuh": "int g();\n"}))
    assert len({a, b, c, d}) == 4


def test_code_only_keeps_literals():
    out = bench._code_only(SRC)
    assert '"a // not a comment"' in out
    assert "'/'" in out
    assert "the header" not in out and "block" not in out and "trailing" not in out
