"""The boundary is a C ABI: include/lqc.h compiles as strict C99, and a C
program links against the built library and calls it (host-only calls, no
device needed): create a DAG, add leaves, a contraction and a term graph,
schedule it and read the figures back."""
import os
import shutil
import subprocess

import pytest

L = pytest.importorskip("paper_2511_02257_b300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include "lqc.h"
int main(void) {
  lqc_dag* d = 0;
  int64_t ext[2] = {3, 3}, a, b, ab, n = 0, roots[1];
  int la[1] = {1}, ra[1] = {0};
  int64_t vo[2] = {0, 2}, vn[2], eo[2] = {0, 2};
  int32_t ed[8] = {0, 1, 1, 0, 0, 0, 1, 1};
  lqc_stats st;
  if (lqc_dag_create(&d, 4, LQC_PREC_FP64) != LQC_OK) return 1;
  if (lqc_dag_add_leaf_tensor(d, 2, ext, 0, &a) != LQC_OK) return 2;
  if (lqc_dag_add_leaf_tensor(d, 2, ext, 0, &b) != LQC_OK) return 3;
  if (lqc_dag_add_contraction(d, a, b, 1, la, ra, &ab) != LQC_OK) return 4;
  vn[0] = a; vn[1] = b;              /* Tr(A B) as a graph */
  if (lqc_dag_add_graphs(d, 1, vo, vn, eo, ed, roots) != LQC_OK) return 5;
  if (lqc_dag_schedule(d, LQC_SCHED_TREE, LQC_EVICT_LRU, 0, &st) != LQC_OK) return 6;
  if (lqc_dag_num_nodes(d, &n) != LQC_OK || n != 4) return 7;
  if (lqc_dag_add_contraction(d, a, b, 1, la, ra, &ab) != LQC_ERR_STATE) return 8;
  printf("%lld %lld %s\n", (long long)st.peak_paper, (long long)st.n_h2d,
         lqc_last_error(d));
  lqc_dag_destroy(d);
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_header_is_c99_and_library_links_from_c(tmp_path):
    src = tmp_path / "abi.c"
    src.write_text(C_SRC)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(L.library_path)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-llqc",
           "-Wl,-rpath," + libdir, "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    peak, n_h2d = (int(x) for x in r.stdout.split()[:2])
    # Tr(A B) over 4 slices of 3x3 complex128: both leaves (2 x 576 B) and
    # the rank-0 root (4 x 16 B, counted in peak_exec only) at the model's peak
    assert n_h2d == 2 and peak == 2 * 4 * 9 * 16
