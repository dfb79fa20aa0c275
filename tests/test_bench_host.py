"""Host-side helpers of bench.py that need no GPU: the code-only hash that ties
a committed ncu summary to the kernel sources it was taken on."""
import bench


def test_comments_and_blank_lines_do_not_count():
    a = "int f(int x) {\n  return x + 1;  // add one\n}\n"
    b = "/* header\n   over two lines */\nint f(int x) {\n\n  return x + 1;\n}\n"
    assert bench.strip_comments(a) == bench.strip_comments(b) == "int f(int x) {\n  return x + 1;\n}"


def test_code_and_literals_count():
    assert bench.strip_comments("int a = 1;") != bench.strip_comments("int a = 2;")
    s = "const char* p = \"a // not a comment /* nor this */\"; char c = '/';"
    assert bench.strip_comments(s) == s
    q = r'const char* q = "say \"//\" twice"; int y;'
    assert bench.strip_comments(q + "  // gone") == q


def _fake_tree(tmp_path, monkeypatch, code):
    csrc = tmp_path / "paper_1104_1824_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(code)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return csrc / "k.cu"


def test_profiled_traffic_follows_the_code(tmp_path, monkeypatch):
    src = _fake_tree(tmp_path, monkeypatch, "__global__ void k() {}\n")
    prof = tmp_path / "profiles" / "expand_kernel_w.txt"
    prof.write_text(f"# summary\nkernel_source_hash: {bench.kernel_source_hash()}\ndram_bytes_per_candidate: 12.5\n")
    assert bench.profiled_traffic("w") == {"bytes_per_candidate": 12.5}
    src.write_text("// the kernel\n__global__ void k() {}  // empty\n\n")
    assert bench.profiled_traffic("w") == {"bytes_per_candidate": 12.5}
    src.write_text("__global__ void k() { int x = 0; }\n")
    assert bench.profiled_traffic("w") is None
    assert bench.profiled_traffic("other") is None


def test_roofline_of_the_packed_store(tmp_path, monkeypatch):
    """The packed form's roofline: its own ncu summary for traffic, the row
    width in the kernel's name, achieved = algorithmic bytes / kernel time,
    against the measured copy bandwidth."""
    import types
    _fake_tree(tmp_path, monkeypatch, "__global__ void k() {}\n")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 5000.0}')
    h = bench.kernel_source_hash()
    (tmp_path / "profiles" / "expand_packed_kernel_w.txt").write_text(
        f"kernel_source_hash: {h}\ndram_bytes_per_candidate: 64.0\n")
    (tmp_path / "profiles" / "expand_kernel_w.txt").write_text(
        f"kernel_source_hash: {h}\ndram_bytes_per_candidate: 256.0\n")
    args = types.SimpleNamespace(workload="w")
    system = types.SimpleNamespace(m=64, R=160)
    r = dict(ms=10.0, expand_ms=5.0, chunks=4, expand_bytes=10 ** 10, candidates=4000, row_width=1)
    packed = bench.roofline_of(args, system, None, "sparse", r, packed=True)
    plain = bench.roofline_of(args, system, None, "sparse", dict(r, row_width=4))
    assert "1 byte(s) per count" in packed["kernel"] and "byte(s)" not in plain["kernel"]
    assert packed["traffic"] == 64 * 1000 and plain["traffic"] == 256 * 1000
    assert packed["achieved"] == 2000.0 and packed["peak"] == 5000.0 and packed["frac"] == 0.4
    assert packed["algorithmic_bytes_per_launch"] == 10 ** 10 // 4 and packed["expand_share_of_step"] == 0.5


def test_e2e_steps_load_explore_and_read_back_every_time():
    """Every timed e2e step goes through the C ABI from host arrays to a full
    read-back; only the pinned result buffer is sized in an untimed step."""
    import types

    import torch

    import snp_synth

    calls = []

    class FakeLibrary:
        SNP_T_TC_I8, SNP_T_SPARSE_I32, SNP_T_TC_F8 = 1, 0, 2

        def snp_load_system(self, m, *arrays):
            calls.append("load")
            return object()

        def snp_explore_opts_init(self):
            return types.SimpleNamespace()

        def snp_explore(self, h, o):
            calls.append("explore")

        def snp_reachable_count(self, h):
            return 10

        def snp_reachable(self, h, out, n):
            calls.append("read")

        def snp_free(self, h):
            calls.append("free")

    class TorchOnCpu:
        int32 = torch.int32

        class cuda:
            @staticmethod
            def synchronize():
                pass

        @staticmethod
        def empty(shape, dtype, pin_memory):
            calls.append("alloc")
            return torch.empty(shape, dtype=dtype)

    args = types.SimpleNamespace(steps=5, transition="sparse")
    r = bench.bench_e2e(args, snp_synth.random_64(1), bench.WORKLOADS["random64"], FakeLibrary(), TorchOnCpu, None)
    step = ["load", "explore", "read", "free"]
    assert calls == ["load", "explore", "alloc", "read", "free"] + step * 3
    assert r["steps"] == 3 and r["d2h_bytes_per_step"] == 10 * 64 * 4 and r["h2d_bytes_per_step"] > 0
