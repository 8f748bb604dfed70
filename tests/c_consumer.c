/* A plain C99 user of the library's C ABI (include/sgs.h): calls the two model
 * builders, which run on the host, and prints what they wrote as text, one
 * value per line, for the test to compare with the oracle's models.
 * Usage: c_consumer anderson n_bath n_channels U eps_d V t mu
 *        c_consumer 2ck L J t */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sgs.h"

static int print_model(int N, const double* A, const int* idx, const double* val, int nq, double e_const) {
    const int n = 2 * N;
    printf("N %d\n", N);
    printf("e_const %.17g\n", e_const);
    for (int k = 0; k < n; k++)
        for (int l = 0; l < n; l++)
            if (A[(size_t)k * n + l] != 0.0) printf("A %d %d %.17g\n", k, l, A[(size_t)k * n + l]);
    for (int q = 0; q < nq; q++)
        printf("Q %d %d %d %d %.17g\n", idx[4 * q], idx[4 * q + 1], idx[4 * q + 2], idx[4 * q + 3], val[q]);
    return 0;
}

int main(int argc, char** argv) {
    if (argc >= 9 && strcmp(argv[1], "anderson") == 0) {
        const int n_bath = atoi(argv[2]), n_channels = atoi(argv[3]);
        const int n = 4 * (1 + n_channels * n_bath);
        double* A = calloc((size_t)n * n, sizeof(double));
        int idx[4];
        double val[1], e_const = 0.0;
        const int N = sgs_build_anderson(n_bath, n_channels, atof(argv[4]), atof(argv[5]), atof(argv[6]),
                                         atof(argv[7]), atof(argv[8]), A, idx, val, &e_const);
        if (N < 0) { fprintf(stderr, "sgs_build_anderson: %d\n", N); return 2; }
        print_model(N, A, idx, val, 1, e_const);
        free(A);
        return 0;
    }
    if (argc >= 5 && strcmp(argv[1], "2ck") == 0) {
        const int L = atoi(argv[2]);
        const int n = 8 * L;
        double* A = calloc((size_t)n * n, sizeof(double));
        int idx[24 * 4];
        double val[24], e_const = 0.0;
        const int N = sgs_build_2ck(L, atof(argv[3]), atof(argv[4]), A, idx, val, &e_const);
        if (N < 0) { fprintf(stderr, "sgs_build_2ck: %d\n", N); return 2; }
        print_model(N, A, idx, val, 24, e_const);
        free(A);
        return 0;
    }
    /* bad arguments reach the library, which must reject them */
    if (argc >= 2 && strcmp(argv[1], "bad") == 0) {
        double A[16], val[24], e_const;
        int idx[96];
        printf("anderson %d\n", sgs_build_anderson(-1, 1, 1.0, 0.0, 0.5, 1.0, 0.0, A, idx, val, &e_const));
        printf("2ck %d\n", sgs_build_2ck(1, 1.0, 0.5, A, idx, val, &e_const));
        return 0;
    }
    fprintf(stderr, "usage: c_consumer anderson n_bath n_channels U eps_d V t mu | 2ck L J t | bad\n");
    return 1;
}
