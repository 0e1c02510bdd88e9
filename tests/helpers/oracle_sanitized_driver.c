/*
 * Driver that runs the C oracle (compiled into the same program, with
 * AddressSanitizer and UndefinedBehaviorSanitizer) on inputs read from a
 * binary file and writes its outputs to another, so a test can run the
 * oracle's simulation under the sanitizers and compare the results with the
 * regular build.
 *
 * Input file, native byte order:
 *   or_model, int32 N, int32 P, int64 S, int32 ts, int32 noise_per_set,
 *   uint64 seed, int64 p_offset, double dt,
 *   double W[N*N], double L[N*N], double prm[P*OR_NPRM]
 * Output file: double E[P*N*(S/ts)], double I[...], double state[P*8*N],
 *   uint32 status[P], then or_tf_eval of (x_e, x_i) = (0.01, 0.02), W = 10,
 *   E_L = -64 for the excitatory row: double jet[6], double aux[8].
 */
#include "../../oracle/adex_oracle.c"

#include <stdio.h>

static int read_all(FILE* f, void* p, size_t n)
{
    return fread(p, 1, n, f) == n;
}

int main(int argc, char** argv)
{
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 3;
    or_model m;
    int32_t N, P, ts, nps;
    int64_t S, p_offset;
    uint64_t seed;
    double dt;
    if (!read_all(f, &m, sizeof m) || !read_all(f, &N, 4) || !read_all(f, &P, 4) || !read_all(f, &S, 8) ||
        !read_all(f, &ts, 4) || !read_all(f, &nps, 4) || !read_all(f, &seed, 8) || !read_all(f, &p_offset, 8) ||
        !read_all(f, &dt, 8))
        return 4;
    if (N < 1 || P < 1 || ts < 1 || S < 0) return 5;
    double* W = malloc(sizeof(double) * (size_t)N * N);
    double* L = malloc(sizeof(double) * (size_t)N * N);
    double* prm = malloc(sizeof(double) * (size_t)P * OR_NPRM);
    if (!read_all(f, W, sizeof(double) * (size_t)N * N) || !read_all(f, L, sizeof(double) * (size_t)N * N) ||
        !read_all(f, prm, sizeof(double) * (size_t)P * OR_NPRM))
        return 6;
    fclose(f);
    const size_t nser = (size_t)P * N * (size_t)(S / ts);
    double* E = malloc(sizeof(double) * (nser ? nser : 1));
    double* I = malloc(sizeof(double) * (nser ? nser : 1));
    double* st = malloc(sizeof(double) * (size_t)P * 8 * N);
    uint32_t* status = malloc(sizeof(uint32_t) * (size_t)P);
    if (or_simulate(&m, N, W, L, P, prm, dt, S, ts, seed, nps, p_offset, 1, E, I, st, status) != 0) return 7;
    double jetv[6], aux[8];
    or_tf_eval(&m, m.P_e, -64.0, 0.01, 0.02, 10.0, jetv, aux);
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 8;
    fwrite(E, sizeof(double), nser, o);
    fwrite(I, sizeof(double), nser, o);
    fwrite(st, sizeof(double), (size_t)P * 8 * N, o);
    fwrite(status, sizeof(uint32_t), (size_t)P, o);
    fwrite(jetv, sizeof(double), 6, o);
    fwrite(aux, sizeof(double), 8, o);
    fclose(o);
    free(W); free(L); free(prm); free(E); free(I); free(st); free(status);
    return 0;
}
