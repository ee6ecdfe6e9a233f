"""The benchmark's reference arm (the oracle on the host cores) runs without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MBF-sets/s" and d["value"] > 0
    assert d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["steps"] == 2


def test_roofline_rows_of_the_leading_kernels():
    """The roofline rows of the two leading C2 kernels: the sweeps against HBM with
    16 B per swept entry + 32 B per cell and sweep, the emulated trailing update against
    the sustained BF16 peak with the BF16 flops of its slice products (whole tiles of
    8 warps x 36 slice pairs x 2 m16n8k16 MMAs) and its FP64-equivalent rate beside it."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2103_08513_gb300 import MRCM
    from synth.configs import workload
    w = workload("c2")
    sizes = MRCM(w.n, w.edges, w.patch, precision="fp32_ir", allocate=False).sizes
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "fp32_tflops": 80.0,
             "fp64_tflops": 1.0, "fp64_source": "test", "source": "test"}
    swept, steps = 74_000_000, 2
    r = bench.roofline("k_ir_sweep", 2.0 * steps, steps, steps, sizes, swept, "fp32_ir", peaks, sweeps=5)
    want = (16.0 * swept + 32.0 * sizes["n_cells"] * 5) / 2e-3 / 1e9
    assert r["bound"] == "hbm" and abs(r["achieved"] - want) <= 1e-3 * want
    r = bench.roofline("k_ldl_update", 2.0 * steps, 70 * steps, steps, sizes, swept, "fp32_ir", peaks)
    tile = 8 * 36 * 2 * (2 * 16 * 8 * 16)
    assert r["bound"] == "tensor" and r["peak"] == 1700.0 and sizes["ldl_update_tensor_flops"] % tile == 0
    assert abs(r["achieved"] - sizes["ldl_update_tensor_flops"] / 2e-3 / 1e12) <= 1e-3 * r["achieved"]
    v = bench.fp64_equivalent_view(2.0 * steps, steps, sizes, peaks)
    assert abs(v["achieved"] - sizes["ldl_update_flops"] / 2e-3 / 1e12) <= 1e-3 * v["achieved"]
