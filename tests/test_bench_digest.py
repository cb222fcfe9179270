"""The kernel-source digest that ties a profile's DRAM counters to the source they were
taken on ignores comments and blank lines, and nothing else."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_strip_comments_keeps_code_and_strings():
    src = 'int a = 1; // one\n/* block\n comment */ const char *s = "//x /*y*/";\n\n  char q = \'\\\'\';\n'
    out = bench.strip_comments(src)
    assert "one" not in out and "block" not in out
    assert '"//x /*y*/"' in out
    assert "char q = '\\''" in out
    assert "\n\n" not in out


def test_digest_ignores_comments_only(tmp_path, monkeypatch):
    a = tmp_path / "k.cu"
    b = tmp_path / "k2.cu"
    a.write_text("__global__ void k(int *p) {\n  p[0] = 1;  // store\n}\n")
    b.write_text("// a kernel\n__global__ void k(int *p) {\n\n  p[0] = 1;  /* the store */\n}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.source_digest(["k.cu"]) == bench.source_digest(["k2.cu"])
    b.write_text("__global__ void k(int *p) {\n  p[0] = 2;\n}\n")
    assert bench.source_digest(["k.cu"]) != bench.source_digest(["k2.cu"])


def test_profiles_name_their_digest():
    # each committed profile that records traffic names the digest of the source it measured
    pdir = os.path.join(bench.ROOT, "profiles")
    for fn in os.listdir(pdir):
        if fn.endswith(".md"):
            txt = open(os.path.join(pdir, fn)).read()
            if "traffic_bytes_per_launch:" in txt:
                assert "source_digest:" in txt, fn
