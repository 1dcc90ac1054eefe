"""Host logic of bench.py's roofline traffic: a committed ncu summary's DRAM bytes are reported
only while the kernel source it was captured on is unchanged (sha256 of the kernel's region)."""
import hashlib
import os

import bench


SRC = """// unrelated header
// Source-lane variant: one block per item
__device__ void helper() {}
__global__ void k_demo(int* x) {
    x[0] = 1;
}
// after the kernel
__global__ void k_other() {
}
"""


def _write(root, digest):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    os.makedirs(os.path.join(root, "src"), exist_ok=True)
    with open(os.path.join(root, "src", "k.cu"), "w") as f:
        f.write(SRC)
    with open(os.path.join(root, "profiles", "k_demo.md"), "w") as f:
        f.write("# demo\n\ntraffic_bytes_per_launch: 123456\n"
                "source_region: src/k.cu | // Source-lane variant: one block per item | k_demo | sha256 %s\n" % digest)


def test_kernel_region_spans_helpers_to_kernel_end():
    reg = bench.kernel_region(SRC, "// Source-lane variant: one block per item", "k_demo")
    assert reg.startswith("// Source-lane variant")
    assert "helper" in reg and "x[0] = 1;" in reg
    assert "k_other" not in reg and reg.endswith("}\n")


def test_traffic_reported_only_for_matching_source(tmp_path, monkeypatch):
    root = str(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    good = hashlib.sha256(bench.kernel_region(SRC, "// Source-lane variant: one block per item",
                                              "k_demo").encode()).hexdigest()
    _write(root, good)
    assert bench.profiled_traffic("k_demo.md") == 123456.0
    _write(root, "0" * 64)
    assert bench.profiled_traffic("k_demo.md") is None
    assert bench.profiled_traffic("missing.md") is None


def test_committed_near_field_summary_parses():
    """The committed summary carries a traffic figure and a digest line in the expected form."""
    text = open(os.path.join(bench.ROOT, "profiles", "k_p2p_lap_src_traffic_laplace_ico6_81920.md")).read()
    assert "traffic_bytes_per_launch:" in text and "source_region:" in text
