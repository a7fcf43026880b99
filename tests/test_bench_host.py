"""Host-side helpers of bench.py (no GPU)."""
import bench


def _digest(tmp_path, text):
    p = tmp_path / "k.cu"
    p.write_text(text)
    return bench.code_digest(str(p))


def test_code_digest_ignores_comments_and_blank_lines(tmp_path):
    base = 'int f(int x) {\n  return x + 1;  // one\n}\nconst char* s = "a // b";\n'
    edited = ('// header comment\nint f(int x) {\n\n  /* block */ return x + 1;  // two\n}\n'
              'const char* s = "a // b";\n')
    assert _digest(tmp_path, base) == _digest(tmp_path, edited)


def test_code_digest_sees_code_and_string_changes(tmp_path):
    base = 'int f(int x) {\n  return x + 1;\n}\nconst char* s = "a // b";\n'
    assert _digest(tmp_path, base) != _digest(tmp_path, base.replace("x + 1", "x + 2"))
    assert _digest(tmp_path, base) != _digest(tmp_path, base.replace("a // b", "a // c"))
