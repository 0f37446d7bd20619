"""include/ns.h is a C header: a plain C11 program that includes it compiles
with -Wall -Werror, links against libns.so and runs the calls that need no
GPU (status strings, shell counts, argument checks on a NULL context)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "ns.h"

int main(void) {
    ns_run_params p;
    memset(&p, 0, sizeof p);
    p.n = 24; p.ny = 36; p.nz = 48; p.lx = 1.0; p.ly = 1.5; p.lz = 0.75; p.dt = 1e-3;
    ns_ctx *ctx = NULL;
    int bad = 0;
    bad |= ns_nbins(32) != 29;
    bad |= ns_run_nbins(&p) < 1;
    bad |= ns_init(NULL, 1, NS_FP64, NULL, &ctx) != NS_ERR_ARG || ctx != NULL;
    bad |= ns_step(NULL, 1) != NS_ERR_ARG;
    bad |= ns_sync(NULL) != NS_ERR_ARG;
    bad |= ns_set_states(NULL, 0, 1, NULL, 0) != NS_ERR_ARG;
    bad |= ns_energy_spectra(NULL, 0, 1, NULL, 0, NULL, NULL) != NS_ERR_ARG;
    bad |= ns_fft_c2r_noalloc(32, 1, NULL, NULL, NULL) != NS_ERR_ARG;
    bad |= strcmp(ns_status_str(NS_OK), "ok") != 0;
    ns_destroy(NULL);
    printf("%d %d %s\n", ns_nbins(32), ns_run_nbins(&p), ns_status_str(NS_ERR_UNSUPPORTED_N));
    return bad;
}
"""


@pytest.fixture(scope="module")
def lib_path():
    from paper_1003_4322_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        from paper_1003_4322_gb300 import build
        build.build()
    return _native.LIB_PATH


def test_c_program_builds_links_and_runs(tmp_path, lib_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib_path)
    subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lns", "-Wl,-rpath," + libdir],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    nb32, nbrun, msg = out.stdout.split(" ", 2)
    assert int(nb32) == 29 and int(nbrun) >= 1 and msg.strip()
