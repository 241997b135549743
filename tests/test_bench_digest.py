"""The bench's tie between recorded DRAM traffic and kernel code: a profile's
traffic is used only while the code (not the comments) of the kernel's
sources is the code the capture was taken with.  Host logic only."""
import os

import pytest

import bench


def test_source_code_text_drops_comments_and_whitespace_only():
    a = 'int f(int x) {  // add one\n  return x + 1; /* done */\n}\n'
    b = 'int f(int x){\n\treturn x+1;}   // other words\n'
    assert bench.source_code_text(a) == bench.source_code_text(b) == "intf(intx){returnx+1;}"
    assert bench.source_code_text("int y = 2;") != bench.source_code_text("int y = 3;")


def test_source_code_text_keeps_string_literals():
    s = 'const char* p = "a // b /* c */ d"; // gone\n'
    assert bench.source_code_text(s) == 'constchar*p="a // b /* c */ d";'
    esc = 'puts("x\\" // y"); // z\n'
    assert bench.source_code_text(esc) == 'puts("x\\" // y");'


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2509_24063_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    for f in ("batched.cu", "codec.cuh", "tera_device.cuh"):
        (csrc / f).write_text(f"// {f}\nint {f.split('.')[0]}_v = 1;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def write_profile(root, digest, nbytes=6.0e9, records=1.6e7):
    (root / "profiles" / "codec_persistent_kernel_uniform_100m.md").write_text(
        "# capture\n\n"
        f"- kernel source digest: `{digest}`\n"
        f"- DRAM bytes per launch: {int(nbytes)}\n"
        f"- records per launch: {int(records)}\n")


def test_recorded_traffic_follows_the_code(fake_root):
    name = "codec_persistent_kernel"
    d0 = bench.kernel_digest(name)
    assert d0 and len(d0) == 16
    write_profile(fake_root, d0)
    assert bench.recorded_traffic(name, "uniform_100m") == (6.0e9, 1.6e7)
    assert bench.recorded_traffic(name, "blobs_16m") is None  # no profile for it
    src = fake_root / "paper_2509_24063_gb300" / "csrc" / "codec.cuh"
    # a comment changes nothing
    src.write_text(src.read_text() + "// a note\n")
    assert bench.kernel_digest(name) == d0
    assert bench.recorded_traffic(name, "uniform_100m") is not None
    # code does: the recorded traffic no longer applies
    src.write_text(src.read_text() + "int extra = 2;\n")
    assert bench.kernel_digest(name) != d0
    assert bench.recorded_traffic(name, "uniform_100m") is None
    write_profile(fake_root, bench.kernel_digest(name), 7.0e9)
    assert bench.recorded_traffic(name, "uniform_100m") == (7.0e9, 1.6e7)


def test_kernels_without_sources_have_no_digest():
    assert bench.kernel_digest("emit_kernel") is None


def test_committed_profiles_parse():
    # every committed traffic record names the fields the bench reads
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for name in bench.KERNEL_SOURCES:
        path = os.path.join(root, "profiles", f"{name}_uniform_100m.md")
        text = open(path).read()
        for key in ("kernel source digest", "DRAM bytes per launch"):
            assert f"- {key}:" in text, (name, key)
