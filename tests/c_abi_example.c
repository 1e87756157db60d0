/*
 * c_abi_example.c -- the scan library driven from plain C through
 * include/pnscan.h alone (no Python, no PyTorch): eight orbits of a small
 * (x0, theta) grid with the manifold correction and the FLI (arXiv:1802.00147,
 * Secs. 2-3), host buffers, run to t = 200 in two calls.
 *
 * Exit status: 0 on success with the integrals restored (printed), 77 when no
 * CUDA device is present (the call that needs one reports
 * PNSCAN_ERR_NODEVICE), 1 on any other failure.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "pnscan.h"

#define N 8

static int check(int code, const char *what)
{
    if (code != PNSCAN_OK) {
        fprintf(stderr, "%s: %s (%d)\n", what, scan_strerror(code), code);
        exit(code == PNSCAN_ERR_NODEVICE ? 77 : 1);
    }
    return code;
}

int main(void)
{
    double cells[N * 9], beta[N], states[N * 12], integ[N * 6], fli[N], t_stop[N];
    int32_t status[N];
    scan_params p;
    scan_handle *h = NULL;
    scan_summary_t sum;
    int i;

    printf("%s\n", scan_version());
    /* cells: x0, pfac, theta1, phi1, theta2, phi2, beta, chi1, chi2 */
    for (i = 0; i < N; i++) {
        double *c = cells + 9 * i;
        c[0] = 15.0 + 3.0 * i;
        c[1] = 0.9;
        c[2] = c[4] = 0.4 * i;
        c[3] = 0.3;
        c[5] = 1.1;
        c[6] = beta[i] = 1.0 - 0.05 * i;
        c[7] = c[8] = 0.8;
    }
    check(scan_params_default(&p), "scan_params_default");
    p.n = N;
    p.beta_m = beta;
    check(scan_create(&p, &h), "scan_create");
    check(scan_setup(h, cells), "scan_setup");
    check(scan_run(h, NULL, 100.0, 1.0), "scan_run");
    check(scan_run(h, NULL, 200.0, 1.0), "scan_run");
    check(scan_read(h, states, integ, fli, status, t_stop), "scan_read");
    check(scan_summary(h, &sum), "scan_summary");
    for (i = 0; i < N; i++) {
        const double dE = fabs(integ[6 * i + 1] - integ[6 * i]) / fabs(integ[6 * i]);
        printf("orbit %d: status %d t %.0f |r| %.3f dE %.1e FLI %.3f\n", i, (int)status[i], t_stop[i],
               sqrt(states[12 * i] * states[12 * i] + states[12 * i + 1] * states[12 * i + 1] +
                    states[12 * i + 2] * states[12 * i + 2]),
               dE, fli[i]);
        if (status[i] == PNSCAN_ORBIT_DONE && !(dE <= 1e-13)) {
            fprintf(stderr, "orbit %d: energy not restored\n", i);
            return 1;
        }
    }
    printf("summary: %lld orbit-steps, max dE %.1e, max dS %.1e\n", (long long)sum.orbit_steps, sum.max_dE,
           sum.max_dS);
    scan_destroy(h);
    return 0;
}
