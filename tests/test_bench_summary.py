"""bench.py's machine-readable ncu summary (the source of roofline.traffic and of the measured
FP64 operations per update): per-kernel means per launch from an ncu --csv metrics capture."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HEAD = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",'
        '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')


def _row(launch, kernel, grid, metric, value):
    return (f'"{launch}","1","python","h","{kernel}","1","7","(32, 8, 1)","{grid}","0","10.3","Command line profiler '
            f'metrics","{metric}","byte","{value}"\n')


def test_summary_means_per_launch_and_fp64_ops(tmp_path):
    k = "void lbmem::k_step<double, false, 0>(lbmem::StepArgs<double>, const double *, double *)"
    rows = [HEAD, "==PROF== noise line\n"]
    for launch, (r, w, dadd, dmul, dfma) in enumerate(((2e7, 3e6, 5e6, 1e6, 1e6), (2.2e7, 3e6, 5e6, 1e6, 1e6))):
        rows += [_row(launch, k, "(16, 64, 1)", "dram__bytes_read.sum", f"{r:,.0f}"),
                 _row(launch, k, "(16, 64, 1)", "dram__bytes_write.sum", w),
                 _row(launch, k, "(16, 64, 1)", "sm__sass_thread_inst_executed_op_dadd_pred_on.sum", dadd),
                 _row(launch, k, "(16, 64, 1)", "sm__sass_thread_inst_executed_op_dmul_pred_on.sum", dmul),
                 _row(launch, k, "(16, 64, 1)", "sm__sass_thread_inst_executed_op_dfma_pred_on.sum", dfma)]
    rows.append(_row(9, "void lbmem::k_step<double, false, 0>(...)", "(64, 256, 1)", "dram__bytes_read.sum", 5))
    csv_path = tmp_path / "c.csv"
    csv_path.write_text("".join(rows))
    out = tmp_path / "counters.json"
    bench.summarize_ncu(str(csv_path), str(out), "ncu ... python bench.py --profile-case")
    d = json.loads(out.read_text())
    assert d["source_sha256_16"] == bench.kernel_source_sha()
    ks = [v for name, v in d["kernels"].items() if "(16, 64, 1)" in name]
    assert len(ks) == 1 and ks[0]["launches"] == 2 and ks[0]["grid_sites"] == 512 * 512
    assert ks[0]["dram_bytes_per_launch"] == 2.1e7 + 3e6
    assert ks[0]["fp64_ops_per_launch"] == 7e6
    other = [v for name, v in d["kernels"].items() if "(64, 256, 1)" in name][0]
    assert "grid_sites" not in other and other["launches"] == 1
