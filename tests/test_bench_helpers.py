"""Host-side helpers of bench.py (no GPU): the ncu-figure lookup keyed by the kernel source's
md5, the Gram-Schmidt work count, the products' algorithmic bytes, the host page report."""
import hashlib
import os

import pytest
import torch

import bench


def _fake_tree(tmp_path, src_text, lines):
    csrc = tmp_path / "paper_2104_10785_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "gk_matvec.cu").write_text(src_text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k.md").write_text("\n".join(lines) + "\n")
    return hashlib.md5(src_text.encode()).hexdigest()


def test_profiled_traffic_reads_the_line_for_the_current_source(tmp_path, monkeypatch):
    h = _fake_tree(tmp_path, "kernel source\n", [])
    (tmp_path / "profiles" / "k.md").write_text(
        f"roofline-traffic: kernel=kA workload=w1 bytes_per_launch=123456 source_md5={h}\n"
        f"roofline-traffic: kernel=kB workload=w1 ratio=0.9647 source_md5={h}\n"
        f"roofline-traffic: kernel=kA workload=w2 bytes_per_launch=7 source_md5={'0' * 32}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("kA", "w1") == 123456
    assert bench.profiled_traffic("kB", "w1", field="ratio") == pytest.approx(0.9647)
    assert bench.profiled_traffic("kA", "w2") is None  # captured from another source
    assert bench.profiled_traffic("kC", "w1") is None
    # editing the kernel source retires every figure taken from it
    (tmp_path / "paper_2104_10785_gb300" / "csrc" / "gk_matvec.cu").write_text("changed\n")
    assert bench.profiled_traffic("kA", "w1") is None


def test_orth_work_counts_one_pass_per_column_and_entry():
    m, n, K = 7, 5, 4
    fl, by = bench.orth_work(m, n, K, 0, 1)
    # step j: the m-vector against j columns, the n-vector against j + 1; 4 flops per entry
    # and column (dot and update), 16 bytes per entry and column plus 24 per entry
    assert fl == sum(4 * (m * j + n * (j + 1)) for j in range(K))
    assert by == sum(16 * (m * j + n * (j + 1)) + 24 * (m + n) for j in range(K))
    fl2, _ = bench.orth_work(m, n, K, 0, 1, passes=2)
    assert fl2 == 2 * fl
    # a restarted cycle starts after the kept columns
    fl3, _ = bench.orth_work(m, n, K, 2, 2)
    assert fl3 == fl + sum(4 * (m * j + n * (j + 1)) for j in range(2, K))


def test_algorithmic_bytes_of_dense_products():
    A = torch.empty((6, 10), dtype=torch.bfloat16)
    w = {"m": 6, "n": 10, "A": A}
    assert bench.algorithmic_bytes(w, "matvec") == 2 * 60 + 4 * 10 + 16 * 6
    assert bench.algorithmic_bytes(w, "matvec_t") == 2 * 60 + 4 * 6 + 16 * 10


def test_host_page_report_has_the_mode():
    rep = bench.host_page_report()
    assert "thp" in rep
    if os.path.exists("/proc/self/smaps_rollup"):
        assert rep.get("anon_huge_kb", 0) >= 0


def test_rsgd_flops_scale_with_products_and_problems():
    """The Algorithm 4 roofline's FP64 count: the inner solves' share is 2 d1 d2 per product, the
    rest of a step grows with the number of problems."""
    w = dict(P=4, d1=784, d2=256, r=5, b=256)
    inner, step = bench.rsgd_flops(w, 10)
    assert inner == 2.0 * 784 * 256 * 10
    inner2, step2 = bench.rsgd_flops(dict(w, P=8), 20)
    assert inner2 == 2 * inner and step2 == 2 * step
    # the mini-batch gradient dominates the rest: 2 b d1 d2 per problem
    assert step > 4 * 2 * 256 * 784 * 256


def test_err_rel_from_residuals_matches_the_oracles_definition():
    """err_rel_paper (from the per-triplet residuals gk_residuals returns) equals the oracle's
    err_rel of Section 5 computed from the factors themselves."""
    import numpy as np

    import bench
    import oracle

    g = np.random.default_rng(5)
    A = g.standard_normal((40, 25))
    U0, s0, Vt0 = np.linalg.svd(A, full_matrices=False)
    k = 6
    U, V = U0[:, :k], Vt0[:k].T
    S = s0[:k] * (1 + 1e-3 * g.standard_normal(k))  # perturbed values: err_rel > 0
    r_atu = np.linalg.norm(A.T @ U - V * S, axis=0)
    got = bench.err_rel_paper(r_atu, S)
    want = oracle.err_rel(oracle.Operator.dense(A), U, S, V)
    assert want > 1e-6
    np.testing.assert_allclose(got, want, rtol=1e-12)
