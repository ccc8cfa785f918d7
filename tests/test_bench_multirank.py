"""The benchmark's multi-rank bookkeeping on CPU: two gloo ranks (one process
each, as torchrun would start them) take the maximum of their timings, and
the whole-job value counts every rank's work over the slowest rank's time.
The reference arm prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    my_ms = [120.0, 150.0][rank]
    mx = bench.max_over_ranks(my_ms, dist, "cpu")
    dist.barrier()
    out[rank] = (mx, bench.whole_job_gups(512 ** 3 * 496, 5, world, mx))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 150.0
    expect = 512 ** 3 * 496 * 5 * 2 / 0.150 / 1e9
    assert out[0][1] == pytest.approx(expect)


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--L", "16",
                        "--steps", "1", "--warmup", "3", "--ref-proj", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--L", "16",
                        "--steps", "1", "--warmup", "3", "--ref-proj", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GUP/s" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1


def test_ncu_traffic_reads_the_committed_summary():
    """The roofline's traffic comes from the committed ncu summary of the
    default kernel while its source is unchanged (the summary records the
    source's sha256)."""
    import hashlib
    import bench
    src = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1104_5243_gb300", "csrc",
                       "bp_tma.cu")
    text = open(os.path.join(os.path.dirname(src), "..", "..", "profiles", "bp_tma_kernel_f32_512.md")).read()
    current = hashlib.sha256(open(src, "rb").read()).hexdigest() in text
    t = bench.ncu_traffic("bp_tma.cu", "bp_tma_kernel_f32_512.md")
    assert (t is not None and t > 1e9) if current else t is None


@pytest.mark.parametrize("L", [1, 7, 8, 64, 100, 512, 1024])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_z_slabs_partition_the_volume(L, world):
    """The ranks' z-slabs tile [0, L) in rank order without gaps or overlap,
    start on multiples of the 8-slice granule, and differ in size by at most
    one granule (Sect. 6's static split of the z loop)."""
    sys.path.insert(0, ROOT)
    import bench
    slabs = [bench.slab_of_rank(L, world, r) for r in range(world)]
    z = 0
    for z0, nz in slabs:
        assert z0 == z and nz >= 0 and (nz == 0 or z0 % 8 == 0)
        z += nz
    assert z == L
    full = [nz for z0, nz in slabs if z0 + nz < L]          # slabs below the top one
    if full:
        assert max(full) - min(full) <= 8
    if world <= -(-L // 8):
        assert all(nz > 0 for _, nz in slabs)


def test_z_slab_split_rejects_bad_arguments():
    sys.path.insert(0, ROOT)
    import bench
    for args in [(0, 1, 0), (8, 0, 0), (8, 2, 2), (8, 2, -1)]:
        with pytest.raises(ValueError):
            bench.slab_of_rank(*args)


def _rank_main_z(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    z0, nz = bench.slab_of_rank(512, world, rank)
    my_ms = [80.0, 90.0][rank]
    mx = bench.max_over_ranks(my_ms, dist, "cpu")
    dist.barrier()
    # strong scaling: the job is one 512^3 volume, whatever the rank count
    out[rank] = (z0, nz, mx, bench.whole_job_gups(512 ** 3 * 496, 5, 1, mx))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_one_volume_by_z_slabs():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main_z, args=(world, port, out), nprocs=world, join=True)
    assert (out[0][0], out[0][1]) == (0, 256) and (out[1][0], out[1][1]) == (256, 256)
    assert out[0][2] == out[1][2] == 90.0
    assert out[0][3] == pytest.approx(512 ** 3 * 496 * 5 / 0.090 / 1e9)


def test_adjoint_roofline_bounds():
    """The adjoint's roofline comes from the method's work alone: FP32 pipe
    at 20.5 operations per update, four conflict-free shared-memory atomics
    per update (one wavefront per SM per clock), one reciprocal per update.
    The measured instruction and wavefront counts stay diagnostics."""
    sys.path.insert(0, ROOT)
    import bench
    b = bench.adjoint_roofline_gups(2000.0, 100)
    assert b["fp32_pipe"] == pytest.approx(100 * 128 / 20.5 * 2.0)
    assert b["smem_atomics"] == pytest.approx(100 * 2.0 * 32 / 4)
    assert b["mufu"] == pytest.approx(100 * 16 * 2.0)
    assert b["min"] == min(b["fp32_pipe"], b["smem_atomics"], b["mufu"])
    d = bench.adjoint_diagnostics_gups(2000.0, 100)
    assert d["issue_at_measured_instr"] == pytest.approx(100 * 128 / bench.ADJ_INSTR_PER_UPDATE * 2.0)
    assert d["smem_atomics_at_measured_wavefronts"] == pytest.approx(
        100 * 2.0 * 32 / (4 * bench.ADJ_ATOMIC_WAVEFRONTS))


def test_forward_roofline_is_the_methods_work():
    """The backprojection's peak at 152 SMs and 2070 MHz: FP32 pipe at 20.5
    operations per update (1965 GUP/s) binds both storage forms on the TMA
    path; shared memory at 16 B (f32) or 8 B (16-bit) per update and MUFU are
    looser.  No kernel-measured count enters the peak, so instructions the
    kernel adds cannot raise it."""
    sys.path.insert(0, ROOT)
    import bench
    for form, smem in (("f32", 16), ("f16", 8), ("bf16", 8)):
        b = bench.roofline_peak_gups("tma", form, 2070.0, 152, 0.0)
        assert b["fp32_pipe"] == pytest.approx(152 * 128 / 20.5 * 2.07)
        assert b["smem"] == pytest.approx(152 * 128 / smem * 2.07)
        assert b["mufu"] == pytest.approx(152 * 16 * 2.07)
        assert b["min"] == pytest.approx(1965.0, rel=1e-3)
        assert "issue" not in b
    t = bench.roofline_peak_gups("texture", "f32", 2070.0, 152, 2.54)
    assert t["min"] == pytest.approx(t["gather"]) and t["gather"] == pytest.approx(152 * 2.54 * 2.07)
    d = bench.roofline_diagnostics_gups("tma", "f32", 2070.0, 152)
    assert d["issue_at_measured_instr"] == pytest.approx(152 * 128 / bench.INSTR_PER_UPDATE[("tma", "f32")] * 2.07)


def test_ncu_fields_need_every_name_and_the_current_source(tmp_path, monkeypatch):
    """A summary's numbers count only with every requested name present and
    the recorded sha256 of the kernel source equal to the current one."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    root = tmp_path
    (root / "profiles").mkdir()
    (root / "paper_1104_5243_gb300" / "csrc").mkdir(parents=True)
    (root / "paper_1104_5243_gb300" / "csrc" / "k.cu").write_bytes(b"kernel source")
    sha = hashlib.sha256(b"kernel source").hexdigest()
    (root / "profiles" / "p.md").write_text(f"text\n\n- fma_pipe_pct: 46.3\n- dram_pct: 6.7\n- source_sha256: {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.ncu_fields("k.cu", "p.md", ["fma_pipe_pct", "dram_pct"]) == {"fma_pipe_pct": 46.3, "dram_pct": 6.7}
    assert bench.ncu_fields("k.cu", "p.md", ["fma_pipe_pct", "smem_wavefronts_pct"]) is None
    (root / "paper_1104_5243_gb300" / "csrc" / "k.cu").write_bytes(b"changed")
    assert bench.ncu_fields("k.cu", "p.md", ["fma_pipe_pct"]) is None


def test_hbm_peak_prefers_the_measured_file(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak_gbs() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6786.2}))
    assert bench.hbm_peak_gbs() == (6786.2, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("{}")
    assert bench.hbm_peak_gbs() == (6800.0, "fallback")


def test_algorithmic_bytes_of_a_launch():
    """Bytes one mid-step launch must move (the roofline's unit): the volume
    read and written once, each projection's staged image once (8-byte
    elements, 1250 columns: float32 pairs over 960 rows, 16-bit column quads
    over 961), and for f32 the 48-byte centring record of every computed
    (brick, projection) pair (bricks of 32 x 16 x depth)."""
    sys.path.insert(0, ROOT)
    import bench
    L, n, isx, isy = 512, 64, 1248, 960
    bricks16 = 16 * 32 * 32
    f32 = bench.algorithmic_bytes(L, n, isx, isy, "f32", "tma", 0.75)
    assert f32 == 8 * L ** 3 + n * 1250 * isy * 8 + int(48 * n * bricks16 * 0.75)
    f32_8 = bench.algorithmic_bytes(L, n, isx, isy, "f32", "tma", 0.75, depth=8)
    assert f32_8 == 8 * L ** 3 + n * 1250 * isy * 8 + int(48 * n * 2 * bricks16 * 0.75)
    f16 = bench.algorithmic_bytes(L, n, isx, isy, "f16", "tma", 0.75)
    assert f16 == 8 * L ** 3 + n * 1250 * (isy + 1) * 8
    # a z-slab of 64 slices: an eighth of the volume and of the bricks
    slab = bench.algorithmic_bytes(L, n, isx, isy, "f32", "tma", 0.75, Lz=64)
    assert slab == 8 * L * L * 64 + n * 1250 * isy * 8 + int(48 * n * (bricks16 // 8) * 0.75)
    tex = bench.algorithmic_bytes(L, n, isx, isy, "f32", "texture", 1.0)
    assert tex == 8 * L ** 3 + n * isx * isy * 4 + 48 * n * (16 * 64 * 128)
    # the diagnostic shared-memory bytes per update: loads plus box fill
    assert bench.tma_smem_bytes_per_update("f32", 16) == pytest.approx(16 + 120 * 58 * 8 / 8192)
    assert bench.tma_smem_bytes_per_update("f16", 8) == pytest.approx(8 + 120 * 35 * 8 / 4096)
