"""The C-ABI library builds, loads and exports every symbol include/uotk.h
declares; host-side validation runs without a GPU.  CPU only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_13618_gb300 import build, uotk
    build.build()
    return uotk.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "uotk.h")).read()
    return sorted(set(re.findall(r"\b(uotk_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("uotk_kernel_sum", "uotk_uot_sinkhorn", "uotk_sinkhorn_divergence", "uotk_mmd2"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_names_match_header(lib):
    from paper_2306_13618_gb300 import uotk
    assert sorted(uotk.EXPORTED) == declared_symbols()


def test_null_context_is_rejected_on_host(lib):
    st = lib.uotk_kernel_sum(None, None, 3, None, 0, None, None, 0, None, 1.0, None)
    assert st == 1  # UOTK_ERR_INVALID, no device touched
    assert lib.uotk_status_string(1) == b"invalid argument"
    assert lib.uotk_status_string(6) == b"not converged"
    assert lib.uotk_launch_count(None) == 0


PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "uotk.h"
#define F(T, f) printf(#T "." #f " %zu %zu\n", offsetof(T, f), sizeof(((T*)0)->f))
int main(void) {
  printf("sizeof.uotk_sum_opts %zu\n", sizeof(uotk_sum_opts));
  printf("sizeof.uotk_nfft_plan_info %zu\n", sizeof(uotk_nfft_plan_info));
  F(uotk_sum_opts, method); F(uotk_sum_opts, grid); F(uotk_sum_opts, bandwidth);
  F(uotk_sum_opts, cutoff); F(uotk_sum_opts, period); F(uotk_sum_opts, target_err);
  F(uotk_sum_opts, kernel); F(uotk_sum_opts, reg_degree);
  F(uotk_nfft_plan_info, d); F(uotk_nfft_plan_info, grid); F(uotk_nfft_plan_info, bandwidth);
  F(uotk_nfft_plan_info, cutoff); F(uotk_nfft_plan_info, center); F(uotk_nfft_plan_info, inv_h);
  F(uotk_nfft_plan_info, h); F(uotk_nfft_plan_info, eps);
  printf("const UOTK_OK %d\nconst UOTK_ERR_NOT_CONVERGED %d\n", UOTK_OK, UOTK_ERR_NOT_CONVERGED);
  printf("const UOTK_DIRECT %d\nconst UOTK_NFFT %d\n", UOTK_DIRECT, UOTK_NFFT);
  printf("const UOTK_DIRECT_BF16 %d\nconst UOTK_DIRECT_BF16X3 %d\n", UOTK_DIRECT_BF16,
         UOTK_DIRECT_BF16X3);
  printf("const UOTK_REF_PRODUCT %d\nconst UOTK_REF_COUNTING %d\n", UOTK_REF_PRODUCT,
         UOTK_REF_COUNTING);
  printf("const UOTK_KERNEL_GAUSS %d\nconst UOTK_KERNEL_LAPLACE %d\n", UOTK_KERNEL_GAUSS,
         UOTK_KERNEL_LAPLACE);
  printf("const UOTK_KERNEL_IMQ %d\nconst UOTK_KERNEL_ENERGY %d\n", UOTK_KERNEL_IMQ,
         UOTK_KERNEL_ENERGY);
  printf("const UOTK_WARM_START %u\nconst UOTK_LOG_DOMAIN %u\nconst UOTK_CSTAR_INIT %u\n",
         UOTK_WARM_START, UOTK_LOG_DOMAIN, UOTK_CSTAR_INIT);
  return 0;
}
"""


def test_struct_layouts_and_constants_match_header(tmp_path):
    """The ctypes mirrors of the header's structs, enums and flags, against a C
    program compiled with the header (plain gcc, no GPU)."""
    import subprocess

    from paper_2306_13618_gb300 import uotk
    src, exe = tmp_path / "probe.c", tmp_path / "probe"
    src.write_text(PROBE)
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    c = {}
    for line in out.splitlines():
        f = line.split()
        if f[0] == "const":
            c["const " + f[1]] = [int(f[2])]
        else:
            c[f[0]] = [int(v) for v in f[1:]]
    assert c["sizeof.uotk_sum_opts"] == [ctypes.sizeof(uotk.SumOpts)]
    assert c["sizeof.uotk_nfft_plan_info"] == [ctypes.sizeof(uotk.NfftPlan)]
    for cls, cname in ((uotk.SumOpts, "uotk_sum_opts"), (uotk.NfftPlan, "uotk_nfft_plan_info")):
        for name, _ in cls._fields_:
            f = getattr(cls, name)
            assert c[f"{cname}.{name}"] == [f.offset, f.size], (cname, name)
    py = {"UOTK_OK": uotk.UOTK_OK, "UOTK_ERR_NOT_CONVERGED": uotk.UOTK_ERR_NOT_CONVERGED,
          "UOTK_DIRECT": uotk.DIRECT, "UOTK_NFFT": uotk.NFFT,
          "UOTK_DIRECT_BF16": uotk.DIRECT_BF16, "UOTK_DIRECT_BF16X3": uotk.DIRECT_BF16X3,
          "UOTK_REF_PRODUCT": uotk.REF_PRODUCT, "UOTK_REF_COUNTING": uotk.REF_COUNTING,
          "UOTK_KERNEL_GAUSS": uotk.KERNELS["gauss"], "UOTK_KERNEL_LAPLACE": uotk.KERNELS["laplace"],
          "UOTK_KERNEL_IMQ": uotk.KERNELS["imq"], "UOTK_KERNEL_ENERGY": uotk.KERNELS["energy"],
          "UOTK_WARM_START": uotk.WARM_START, "UOTK_LOG_DOMAIN": uotk.LOG_DOMAIN,
          "UOTK_CSTAR_INIT": uotk.CSTAR_INIT}
    for k, v in py.items():
        assert c["const " + k] == [v], k


def test_binding_argument_checks_on_host():
    """Arguments the binding refuses before any library call: host tensors,
    other dtypes, point arrays of the wrong rank; 1-D points are one column."""
    torch = pytest.importorskip("torch")
    from paper_2306_13618_gb300 import uotk
    with pytest.raises(TypeError):
        uotk._f32(torch.zeros(4), "w")                       # host memory
    with pytest.raises(TypeError):
        uotk._f32(torch.zeros(4, dtype=torch.float64), "w")  # FP64
    o = uotk._opts("nfft", grid=64, cutoff=5, target_err=1e-4, kernel="imq", reg_degree=6)
    assert (o.method, o.grid, o.cutoff, o.kernel, o.reg_degree) == (uotk.NFFT, 64, 5, 2, 6)
    assert o.target_err == 1e-4 and o.period == 0.0 and o.bandwidth == 0
    d = uotk._opts()
    assert (d.method, d.kernel) == (uotk.DIRECT, 0)
    assert uotk._opts("direct_bf16x3").method == uotk.DIRECT_BF16X3
