"""Host-side helpers of bench.py (no GPU): the DRAM-traffic record that fills
the roofline line's "traffic" field is used only while the kernel source it
was measured on is unchanged, and its split-K adjustment adds the partials of
the extra splits."""
import hashlib
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _tree(tmp_path, tc_src=b"kernels", ptx_src=b"wrappers"):
    csrc = tmp_path / "paper_2407_12168_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "ensf_tc.cu").write_bytes(tc_src)
    (csrc / "ensf_ptx.cuh").write_bytes(ptx_src)
    (csrc / "ensf_simt.cu").write_bytes(b"simt")
    (tmp_path / "profiles").mkdir()
    return hashlib.sha256(tc_src + ptx_src).hexdigest()[:16]


def test_traffic_record_needs_the_measured_source(tmp_path):
    b = _bench()
    sha = _tree(tmp_path)
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(
        f"traffic gram_pair large-512 split-bf16 {sha} bytes_per_launch=4298000000 splits=4\n"
        f"traffic wx_em_staged large-512 split-bf16 {sha} bytes_per_launch=7110000000\n"
        "traffic wx_em_slice large-512 split-bf16 0123456789abcdef bytes_per_launch=1\n")
    b.ROOT = str(tmp_path)
    # the recorded figure, and the partials of 5 more splits at N = 1024 added
    assert b._traffic_record("gram_pair", "large-512", "split-bf16", 4, 1024) == 4298000000
    assert b._traffic_record("gram_pair", "large-512", "split-bf16", 9, 1024) == 4298000000 + 5 * 1024 * 1024 * 4
    assert b._traffic_record("wx_em_staged", "large-512", "split-bf16") == 7110000000
    # another source hash, workload or path: no figure
    assert b._traffic_record("wx_em_slice", "large-512", "split-bf16") is None
    assert b._traffic_record("gram_pair", "medium-192", "split-bf16", 4, 1024) is None
    assert b._traffic_record("gram_pair", "large-512", "fp32", 4, 1024) is None
    # an edit of the kernel file invalidates the record
    (tmp_path / "paper_2407_12168_gb300" / "csrc" / "ensf_tc.cu").write_bytes(b"kernels, changed")
    assert b._traffic_record("wx_em_staged", "large-512", "split-bf16") is None


def test_traffic_record_absent_file(tmp_path):
    b = _bench()
    _tree(tmp_path)
    b.ROOT = str(tmp_path)
    assert b._traffic_record("gram_pair", "large-512", "split-bf16", 4, 1024) is None


def test_committed_traffic_lines_parse():
    """Every traffic line of the committed record has the fields the bench reads."""
    import re
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    lines = [ln for ln in open(path) if ln.startswith("traffic ")]
    assert lines
    pat = re.compile(r"^traffic\s+(\S+)\s+(\S+)\s+(\S+)\s+([0-9a-f]{16})\s+bytes_per_launch=(\d+)(?:\s+splits=(\d+))?\s*$")
    tags = {pat.match(ln).group(1) for ln in lines}
    assert {"gram_pair", "gram_pair_noise", "wx_em_staged", "wx_em_slice"} <= tags


def test_cpu_nodes_lists_nodes_or_none():
    b = _bench()
    nodes = b._cpu_nodes()
    assert nodes is None or all(isinstance(v, int) and v >= 0 for v in nodes)
