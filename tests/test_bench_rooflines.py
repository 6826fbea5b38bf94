"""The bench line's roofline objects (CPU): achieved rates from the algorithmic work per launch of
vortex256 divided by the live average launch time, fractions of the stated peaks, the dominant
kernel by total time, and traffic taken only from the ncu figures captured for that workload."""

import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

bench = pytest.importorskip("bench")

PROF = {"gmres": (16.2, 2), "condense_factor": (10.8, 2), "condense_products": (8.0, 2), "jacobian": (10.9, 2)}
STATS = {"gmres_iterations": 36, "newton_iterations": 2}
PEAKS = {"hbm_gbs": 6779.0, "bf16_tflops": 1933.0}
CLOCKS = {"sm_max_mhz": 2070.0}


def _vortex256():
    return SimpleNamespace(mesh=SimpleNamespace(nelem=65536), p=4)


def test_gmres_cycle_rate_and_dominant_kernel():
    dom, out = bench.kernel_rooflines(PROF, STATS, _vortex256(), PEAKS, CLOCKS, "vortex256", 2)
    assert dom == "gmres"
    g = out["gmres"]
    # algorithmic bytes of one 18-iteration cycle: per iteration the S blocks 65 536 x 80 x 80 x 4 B and
    # the gathered and scattered FP64 trace values 65 536 x 2 x 80 x 8 B; at iteration k the
    # orthogonalisation's (k + 2) x 2 621 440 x 8 B
    alg = 18 * (65536 * 6400 * 4 + 65536 * 2 * 80 * 8) + sum((k + 2) * 2621440 * 8 for k in range(1, 19))
    assert g["algorithmic_bytes"] == alg
    assert abs(alg - 36.05e9) < 0.01e9  # about 36 GB per launch
    # what the implementation moves beyond those is reported apart: the face-block inverses and the
    # second Gram-Schmidt pass over the FP32 basis
    assert g["implementation_extra_bytes"] == 18 * 131072 * 400 * 4 + sum((k + 1) * 2621440 * 4 for k in range(1, 19))
    achieved = alg / 8.1e-3 / 1e9
    assert g["unit"] == "GB/s" and g["bound"] == "hbm"
    assert abs(g["achieved"] - achieved) < 1e-6 * achieved
    assert abs(g["frac"] - achieved / 6779.0) < 1e-9
    # traffic: the captured DRAM bytes per element and iteration (vortex128p4, 16 384 elements, 60
    # iterations, 31.28 GB) times this launch's 65 536 elements and 18 iterations, about 1.04 x alg
    assert g["traffic"] == pytest.approx(31279474432 / (16384 * 60) * 65536 * 18)
    assert 1.0 < g["traffic"] / alg < 1.1
    assert g["avg_launch_ms"] == pytest.approx(8.1)


def test_element_kernels_use_the_captured_traffic_of_their_workload():
    _, out = bench.kernel_rooflines(PROF, STATS, _vortex256(), PEAKS, CLOCKS, "vortex256", 2)
    table = bench.NCU_TRAFFIC_BYTES["vortex256"]
    assert out["jacobian"]["traffic"] == table["k_jacobian"]
    assert out["condense_factor"]["kernel"] == "k_inverse_tc"
    assert out["condense_factor"]["traffic"] == table["k_inverse_tc"]
    # the products are HBM-bound here: 187 KB per element in 4 ms is a larger fraction of the copy
    # bandwidth than 2.9 MFLOP per element is of the TF32 roof
    p = out["condense_products"]
    assert p["bound"] == "hbm" and p["traffic"] == table["k_products_tc"]
    by = 65536 * (4.0 * (100 * 100 + 2 * 100 * 80 + 80 * 80) + 4.0 * (100 * 80 + 80 * 80)) / 4.0e-3 / 1e9
    assert abs(p["achieved"] - by) < 1e-6 * by
    # FP32 roof: 152 SMs x 256 flop per clock x 2070 MHz
    j = out["jacobian"]
    assert abs(j["peak"] - 152 * 256 * 2070e6 / 1e12) < 1e-9
    flops = 65536 * (100 + 80) ** 2 * (2 * 5 + 4) * 2.0 / 5.45e-3 / 1e12
    assert abs(j["achieved"] - flops) < 1e-6 * flops


def test_no_traffic_without_a_capture_and_fma_kernel_names():
    _, out = bench.kernel_rooflines(PROF, STATS, _vortex256(), PEAKS, CLOCKS, "vortex64", 0)
    # per-launch element-kernel traffic is taken only from the captures of the named workload; the
    # GMRES cycle's comes from its per element-iteration figure for the block shape (nT = 80 here)
    assert all(v["traffic"] is None for k, v in out.items() if k != "gmres")
    assert out["gmres"]["traffic"] is not None
    assert out["condense_factor"]["kernel"] == "k_inverse_rq"
    assert out["condense_products"]["kernel"] == "k_products_x+k_products_s"
    _, out = bench.kernel_rooflines(PROF, STATS, _vortex256(), PEAKS, CLOCKS, "vortex256", 3)
    assert out["condense_factor"]["kernel"] == "k_inverse_tc"


def test_measured_pipe_peaks_replace_the_derived_ones():
    peaks = dict(PEAKS, fp32_tflops_measured=70.0, tf32_tflops_measured=900.0)
    _, out = bench.kernel_rooflines(PROF, STATS, _vortex256(), peaks, CLOCKS, "vortex256", 2)
    assert out["jacobian"]["peak"] == 70.0 and "fr_measure_peak" in out["jacobian"]["peak_source"]
    assert out["condense_factor"]["peak"] == 70.0
