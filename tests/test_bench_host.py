"""Host logic of bench.py's roofline bookkeeping, on CPU: the DRAM traffic of the dominant
kernel is reported only while the kernel's source is the one the capture was taken on."""
import bench


def _profile(tmp_path, nbytes, sha):
    p = tmp_path / "capture.md"
    p.write_text("# capture\n\ntraffic_bytes_per_launch: %d\nsource_sha256_16: %s\n" % (nbytes, sha))
    return str(p)


def test_matching_source_reports_the_bytes(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(src))
    got, note = bench.recorded_traffic(_profile(tmp_path, 5660805888, bench.source_sha(str(src))))
    assert got == 5660805888
    assert "ncu capture" in note


def test_changed_source_reads_as_stale(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(src))
    prof = _profile(tmp_path, 123, bench.source_sha(str(src)))
    src.write_text("__global__ void k() { /* changed */ }\n")
    got, note = bench.recorded_traffic(prof)
    assert got is None and note.startswith("stale")


def test_missing_or_incomplete_capture(tmp_path):
    got, note = bench.recorded_traffic(str(tmp_path / "absent.md"))
    assert got is None and "no capture" in note
    p = tmp_path / "partial.md"
    p.write_text("traffic_bytes_per_launch: 1\n")
    got, note = bench.recorded_traffic(str(p))
    assert got is None and "no capture recorded" in note

