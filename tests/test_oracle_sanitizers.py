"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU).

A small C driver, compiled here with the oracle's source and
-fsanitize=address,undefined, runs an ensemble through initialisation, steps
with and without flow, a decision tape recorded and replayed, the correlator
(all channels) and the stress logs, and reads every accessor back.  Any
sanitizer report makes it exit non-zero.
"""
import os
import shutil
import subprocess

import pytest

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

DRIVER = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "ss_oracle.h"

int main(void) {
    or_params p;
    memset(&p, 0, sizeof(p));
    p.N = 24; p.z_max = 24; p.N0 = 4.0; p.Ns = 0.5; p.zeta_s = 0.1; p.dt = 0.01;
    p.b = 1.0; p.kT = 1.0; p.zeta = 1.0;
    or_params_derive(&p);
    const int M = 37, G = 4, L = 10, nlog = 8;
    or_ens* e = or_ens_create(&p, 99, M, 5, G, L, 25, nlog);
    if (!e) return 2;
    or_ens_init(e);
    double kap[9] = {0, 0.1, 0, 0, 0, 0, 0, 0, 0};
    or_ens_set_flow(e, 50, kap);
    if (or_ens_run(e, 100, 2, NULL, NULL, NULL) != 0) return 3;
    unsigned char* tape = (unsigned char*)calloc((size_t)60 * M * p.N, 1);
    double* R = (double*)malloc(sizeof(double) * M * p.N * 3);
    double* A = (double*)malloc(sizeof(double) * M * p.z_max * 3);
    int* Z = (int*)malloc(sizeof(int) * M);
    int* S = (int*)malloc(sizeof(int) * M * p.z_max);
    or_ens_get_state(e, R, Z, S, A);
    if (or_ens_run_tape(e, 60, 2, NULL, NULL, NULL, tape, 1) != 0) return 4;
    or_ens_set_state(e, R, Z, S, A);
    or_ens_set_step(e, 100);
    if (or_ens_run_tape(e, 60, 2, NULL, NULL, NULL, tape, 2) != 0) return 5;
    double* acc = (double*)malloc(sizeof(double) * G * L * OR_P * 6);
    double* acc_tt = (double*)malloc(sizeof(double) * G * L * OR_P * 3);
    int64_t n = 0;
    or_ens_corr(e, acc, &n);
    or_ens_corr_tt(e, acc_tt);
    double* logs = (double*)malloc(sizeof(double) * nlog * G * 14);
    int64_t steps[8];
    int k = or_ens_logs(e, logs, steps, nlog);
    int64_t cnt[5];
    or_ens_counters(e, cnt);
    or_ens_reset_obs(e);
    or_ens_destroy(e);
    free(tape); free(R); free(A); free(Z); free(S); free(acc); free(acc_tt); free(logs);
    printf("ok %d %lld %lld\n", k, (long long)n, (long long)cnt[0]);
    return 0;
}
"""


def test_oracle_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no gcc")
    src = tmp_path / "driver.c"
    src.write_text(DRIVER)
    exe = tmp_path / "driver"
    cmd = [cc, "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=all", "-fopenmp", "-I", ORACLE, str(src),
           os.path.join(ORACLE, "ss_oracle.c"), "-lm", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr and "not supported" in r.stderr:
        pytest.skip("sanitizers unavailable")
    assert r.returncode == 0, r.stderr[-2000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", OMP_NUM_THREADS="2")
    run = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, (run.stdout[-1000:], run.stderr[-3000:])
    assert run.stdout.startswith("ok")
