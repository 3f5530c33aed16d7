"""The bench's byte and flop models, the roofline kernel choice and the reference arm's line
(CPU; no device).

The HBM fractions the bench line reports divide a kernel's algorithmic bytes by its measured
launch time, and the roofline sits on the largest-share kernel that has a model.  These tests
hold the models to the fields each kernel streams, as counted from the kernels' arguments
(FP64 fields 8 B, FP32 4 B; a 7-point operator of the Newton matrix carries both couplings of
each face), and check that every kernel the bench reports a fraction for has a model."""
import bench


def test_every_reported_kernel_has_a_byte_model():
    for nonsym in (False, True):
        ab = bench.alg_bytes(nonsym)
        missing = [k for k in bench.LINEAR_KERNELS if k not in ab]
        assert not missing, missing


def test_multigrid_byte_models_count_the_fields():
    sym, ns = bench.alg_bytes(False), bench.alg_bytes(True)
    # sweep: x, b, omega / diag and the face arrays read, x written (3 or 6 face arrays)
    assert sym["mg_smooth_f32_fine"] == 4 * (3 + 3) + 4
    assert ns["mg_smooth_f32_fine"] == 4 * (3 + 6) + 4 == 40
    assert ns["mg_smooth_f64_fine"] == 2 * ns["mg_smooth_f32_fine"]
    # the first sweep reads b and omega / diag only
    assert ns["mg_smooth_f32_fine_first"] == 12
    # restriction: the sweep's reads with diag in place of omega / diag, one value per 8 cells
    assert ns["mg_restrict_f32_fine"] == 4 * (3 + 6) + 0.5
    # prolongation: x read and written, the parent read once per 8 cells
    assert ns["mg_prolong_f32_fine"] == 8.5
    # conversions: one FP64 and one FP32 value per cell
    assert ns["mg_to_f32"] == ns["mg_from_f32"] == 12


def test_krylov_byte_models_count_the_fields():
    ab = bench.alg_bytes(True)
    # y = A x: x, diag, P and Q of 3 faces and the dot's vector read, y written
    assert ab["bicg_matvec"] == 8 * 9 + 8 == 80
    assert ab["bicg_update_p"] == 8 * 3 + 8
    assert ab["bicg_update_s"] == 8 * 2 + 8


def test_dominant_kernel_is_the_largest_modelled_share():
    ab = bench.alg_bytes(True)
    kt = {"krylov_graph": (500.0, 10),               # a graph wrapper: no model
          "cell_residual_schur": (45.0, 4),
          "mg_smooth_f32_fine": (26.0, 228),
          "bicg_matvec": (28.0, 76)}
    assert bench.dominant_kernel(kt, ab) == "cell_residual_schur"
    kt["mg_smooth_f32_fine"] = (60.0, 228)
    assert bench.dominant_kernel(kt, ab) == "mg_smooth_f32_fine"
    assert bench.dominant_kernel({"krylov_graph": (1.0, 1)}, ab) is None


def test_cell_kernel_flop_model_and_peak():
    # 175 DFMA (2 flops) + 106 DMUL + 76 DADD per cell, from the instruction counts
    assert bench.ALU_FLOPS["cell_residual_schur"] == 2 * 175 + 106 + 76
    # 152 SMs x 2070 MHz x 2 DFMA per clock per SM x 2 flops
    assert abs(bench.FP64_PEAK_TFLOPS - 152 * 2.070e9 * 2 * 2 / 1e12) < 1e-9


def test_workload_sources_keep_the_256_cube_density():
    assert bench.workload_sources(256) == 64
    assert bench.workload_sources(128) == 8
    assert bench.workload_sources(64) == 1
    assert bench.workload_sources(48) == 1


def test_reference_arm_prints_the_contract_line(capsys, monkeypatch):
    """`bench.py --impl reference` times the oracle on a sub-box of the same workload and prints
    one JSON line with the bench's keys, `impl` = reference, its own CPU baseline and an e2e
    block without device copies (a tiny sub-box here, to keep the CPU suite short)."""
    import json
    import types
    monkeypatch.setenv("RHI_REF_SAMPLE_N", "8")
    args = types.SimpleNamespace(steps=1, warmup=0, n=256)
    bench.reference_arm(args, 0, 1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
