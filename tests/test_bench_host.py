"""Host-side logic of bench.py, on the CPU: the operation counts behind the
roofline fractions (the planar float and FP64 steps and the 3D form), the
number of our kernel launches a step claims (the ncu launch list of the default
step shows births, amplitude maximum, float pass, three compaction kernels,
group plan, redo and two spectra), the parsing of the sampled SM clocks and throttle
reasons that decides whether a measurement is kept, and the CPU baseline's
all-thread, one-thread and host-model fields."""
import bench
from paper_2601_17164_gb300 import workloads as W


def test_operation_counts_per_trajectory_step():
    # the planar float step follows the branch and folds its action every fifth step
    assert abs(bench.flops_per_traj_step(W.POT_SOFTCORE, planar=True, compensated=True) - 507.4) < 1e-9
    assert bench.flops_per_traj_step(W.POT_SOFTCORE, planar=True, compensated=False) == 471
    assert bench.flops_per_traj_step(W.POT_SOFTCORE, planar=False, compensated=True) == 1253
    for pot in (W.POT_SOFTCORE, W.POT_TONGLIN, W.POT_HARMONIC, W.POT_ZERO):
        # the Kahan terms and the two-float action add work (16 + 2.8 + 48 + 12 in the
        # planar form, where the float pass also follows the branch every fifth step only)
        assert bench.flops_per_traj_step(pot, False, True) > bench.flops_per_traj_step(pot, False, False)
        assert abs(bench.flops_per_traj_step(pot, True, True) - (bench.flops_per_traj_step(pot, True, False) + 78.8 - 0.8 * 53)) < 1e-9
        # the planar form (25 reals) is the cheaper one
        assert bench.flops_per_traj_step(pot, True) < bench.flops_per_traj_step(pot, False)
    # three exponentials per Tong-Lin evaluation against one rsqrt for the soft core
    assert bench.flops_per_traj_step(W.POT_TONGLIN) > bench.flops_per_traj_step(W.POT_SOFTCORE)


def test_launches_per_step():
    n, n_steps = W.H_800_8CYC_1M.n, 88256
    # sequential mixed step: births, amplitude maximum, float pass, count / scan /
    # scatter, group plan, redo, two spectra
    assert bench.launches_per_step(n, n_steps, 1000, 1, True, overlap=2) == 10
    assert bench.launches_per_step(n, n_steps, 1000, 1, False, overlap=2) == 9      # no amplitude floor
    assert bench.launches_per_step(n, n_steps, 1000, 1, True, overlap=2, esc_precision=2) == 9   # one-thread redo
    assert bench.launches_per_step(n, n_steps, 1000, 0, True) == 4                   # FP64: one pass
    # eight birth chunks, each with its float pass, compaction, plan and redo
    assert bench.launches_per_step(n, n_steps, 1000, 1, True, overlap=0) == 2 + 8 * 6 + 2
    # a chunk is at least 64 blocks: 5000 births make one chunk
    assert bench.launches_per_step(5000, n_steps, 1000, 1, True, overlap=0) == 2 + 6 + 2
    # time segments: at most eight, one per window when there are fewer windows
    assert bench.launches_per_step(n, n_steps, 1000, 1, True, overlap=1) == 2 + 8 * 6 + 2
    assert bench.launches_per_step(n, 3000, 1000, 1, True, overlap=1) == 2 + 4 * 6 + 2


class _Exited:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _parse(lines, tmp_path):
    c = bench.Clocks(0)
    p = tmp_path / "clk.csv"
    p.write_text("".join(lines))
    c.path, c.proc = str(p), _Exited()
    return c.stop()


IDLE = "0, 1965, 2070, 110.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
LOAD = "0, 2070, 2070, 385.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
CAPPED = "0, 1800, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
HOT = "0, 1500, 2070, 1200.0, 0x40, Not Active, Active, Not Active, Not Active\n"


def test_clock_samples_and_throttle_reasons(tmp_path):
    r = _parse([IDLE, LOAD, LOAD, LOAD], tmp_path)
    # median over the samples under load (power above 200 W), the idle one left out
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070 and r["reasons"] == [] and r["samples"] == 4
    r = _parse([LOAD, CAPPED, HOT], tmp_path)
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert r["sm_mhz"] == 1800 and r["power_w_max"] == 1390.0
    # a clock lock shows as a low median with no reason active
    r = _parse([IDLE.replace("110.5", "300.0").replace("1965", "990")] * 3, tmp_path)
    assert r["sm_mhz"] == 990 and r["sm_max_mhz"] == 2070 and r["reasons"] == []
    # unreadable rows ([N/A] power, short lines) are skipped
    r = _parse(["0, 2070, 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active\n", "garbage\n", LOAD],
               tmp_path)
    assert r["samples"] == 1
    assert _parse(["garbage\n"], tmp_path)["reasons"] == ["no samples"]
    c = bench.Clocks(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]                          # never started


def test_cpu_baseline_reports_all_threads_one_thread_and_model():
    import oracle as O
    w = W.H_800_2CYC_GRID
    before = O.max_threads()
    r = bench.cpu_baseline(w, 64)
    assert O.max_threads() == before                                                   # restored
    assert r["kind"] == "oracle" and r["cores"] == before and r["value"] > 0
    assert r["one_thread"]["value"] > 0 and r["one_thread"]["unit"] == r["unit"]
    assert isinstance(r["cpu_model"], str) and r["cpu_model"]
