"""CPU checks of bench.py's host logic: the code hash that ties the stored
DRAM traffic of the force kernel to the kernel's code."""
import bench


def test_code_only_drops_comments_and_layout():
    src = ('int a = 1; // one\n/* two\n   lines */  int  b =\n 2;\n'
           'const char *s = "x // not a comment /* nor this */";\n'
           "char q = '\"'; char r = '\\''; // tail\n")
    assert bench.code_only(src) == (
        'int a = 1; int b = 2; const char *s = "x // not a comment /* nor this */"; '
        "char q = '\"'; char r = '\\'';")


def test_code_only_keeps_every_token_of_the_code():
    a = "x = y / z; w = p /q;"
    assert bench.code_only(a) == a
    assert bench.code_only("a/**/b") == "a b"


def test_kernel_hash_ignores_comments_only(tmp_path, monkeypatch):
    f = tmp_path / "k.cu"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ["k.cu"])
    f.write_text("__global__ void k(int *p) { p[0] = 1; }\n")
    h0 = bench.kernel_hash()
    f.write_text("// the kernel\n__global__ void k(int *p)\n{\n    p[0] = 1;  /* store */\n}\n")
    assert bench.kernel_hash() == h0
    f.write_text("__global__ void k(int *p) { p[0] = 2; }\n")
    assert bench.kernel_hash() != h0


def test_cpu_model_names_the_host():
    name = bench.cpu_model()
    assert isinstance(name, str) and name.strip()
