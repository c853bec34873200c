"""Host-side arithmetic of bench.py (no GPU): algorithmic bytes and the derived figures."""
import bench


def test_derived_metrics_from_a_kernel_profile():
    prof = {"factor": {"ms": 228.0886, "launches": 3}, "sptrsv_fwd/t=1": {"ms": 18258.3, "launches": 12543}}
    d = bench.derived_metrics(prof, 1_000_000, 20, 24486.1, 94.59)
    assert abs(d["evals_per_s_incl_graph"] - 1000.0 / (24486.1 + 94.59)) < 1e-15
    f = d["factor_roofline"]
    assert f["bound"] == "alu" and f["unit"] == "TFLOP/s"
    assert abs(f["flops_per_row"] - (20 ** 3 / 3 + 800 + 40)) < 1e-9
    # nnz / m rows-equivalent: (n - m) full rows plus the short leading rows
    rows_eq = bench._nnz(1_000_000, 20) / 20
    assert abs(f["achieved"] - rows_eq * f["flops_per_row"] / (228.0886 / 3 / 1000) / 1e12) < 1e-12
    assert 0 < f["frac"] < 1 and abs(f["peak"] - 1.25856) < 1e-4
    # a profile without the factor class gives only the rate
    assert set(bench.derived_metrics({}, 10, 3, 5.0, 1.0)) == {"evals_per_s_incl_graph"}


def test_nnz_counts_the_short_leading_rows():
    assert bench._nnz(1, 5) == 0
    assert bench._nnz(4, 5) == 0 + 1 + 2 + 3
    assert bench._nnz(10, 3) == 0 + 1 + 2 + 7 * 3


def test_algorithmic_bytes_of_the_streaming_classes():
    n, m, t, e = 1000, 5, 8, 4
    vec = n * t * e
    nnz = bench._nnz(n, m)
    assert bench.algorithmic_bytes("coldot", n, m, t, e) == 2 * vec
    assert bench.algorithmic_bytes("pcg_update", n, m, t, e) == 4.5 * vec
    assert bench.algorithmic_bytes("spmv_B", n, m, t, e) == nnz * (4 + e) + 2 * vec + n * e
    assert bench.algorithmic_bytes("woodbury", n, m, t, e, k=16) == 2 * n * 16 * e + 3 * vec + n * e
