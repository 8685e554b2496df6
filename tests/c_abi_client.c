/* A plain C11 client of the library's C ABI (no Python, no C++): reads a system and a
 * model from a binary file, creates an FP64 system, evaluates energy, forces and fields,
 * advances 10 Langevin steps and writes the results.  Used by tests/test_c_abi.py.
 *
 * input (native little-endian):  int64 n; double box[3]; int32 periodic[3];
 *   int32 n_species, n_ch, l_max, basis_k, n_hidden; double rc_rad, rc_ang, b1;
 *   double coeffs[n_species^2 * 6 * n_ch * basis_k], q_scaler[66], w0[n_hidden * 66],
 *   b0[n_hidden], w1[n_hidden], mass[n_species], moment[n_species];
 *   int32 species[n]; double pos[3n], spins[3n], vel[3n]
 * output: double E0, F0[3n], H0[3n], pos[3n], spins[3n], E1; int64 step
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "spinlat.h"

static void *grab(FILE *f, size_t bytes) {
    void *p = malloc(bytes ? bytes : 1);
    if (!p || fread(p, 1, bytes, f) != bytes) {
        fprintf(stderr, "short input\n");
        exit(2);
    }
    return p;
}

#define CHECK(call)                                                          \
    do {                                                                     \
        int rc_ = (call);                                                    \
        if (rc_ != SL_OK) {                                                  \
            fprintf(stderr, "%s -> %d: %s\n", #call, rc_, sl_last_error()); \
            return 3;                                                        \
        }                                                                    \
    } while (0)

int main(int argc, char **argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s input.bin output.bin\n", argv[0]);
        return 1;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) return 1;
    int64_t n = *(int64_t *)grab(in, sizeof(int64_t));
    double *box = grab(in, 3 * sizeof(double));
    int32_t *periodic = grab(in, 3 * sizeof(int32_t));
    int32_t *dims = grab(in, 5 * sizeof(int32_t));
    double *cuts = grab(in, 3 * sizeof(double));
    sl_nep_params p;
    p.n_species = dims[0];
    p.n_ch = dims[1];
    p.l_max = dims[2];
    p.basis_k = dims[3];
    p.n_hidden = dims[4];
    p.rc_rad = cuts[0];
    p.rc_ang = cuts[1];
    p.b1 = cuts[2];
    const size_t ns = (size_t)p.n_species, nh = (size_t)p.n_hidden;
    p.coeffs = grab(in, ns * ns * 6 * (size_t)p.n_ch * (size_t)p.basis_k * sizeof(double));
    p.q_scaler = grab(in, 66 * sizeof(double));
    p.w0 = grab(in, nh * 66 * sizeof(double));
    p.b0 = grab(in, nh * sizeof(double));
    p.w1 = grab(in, nh * sizeof(double));
    p.mass_amu = grab(in, ns * sizeof(double));
    p.moment_muB = grab(in, ns * sizeof(double));
    int32_t *species = grab(in, (size_t)n * sizeof(int32_t));
    double *pos = grab(in, 3 * (size_t)n * sizeof(double));
    double *spins = grab(in, 3 * (size_t)n * sizeof(double));
    double *vel = grab(in, 3 * (size_t)n * sizeof(double));
    fclose(in);

    sl_options opt;
    sl_default_options(&opt);
    opt.precision = SL_PREC_FP64;
    sl_system *sys = NULL;
    CHECK(sl_create_system(pos, spins, box, periodic, species, n, vel, &p, &opt, &sys));
    double *F = malloc(3 * (size_t)n * sizeof(double)), *H = malloc(3 * (size_t)n * sizeof(double));
    double E0 = 0.0, E1 = 0.0;
    CHECK(sl_energy_forces_fields(sys, &E0, F, H, NULL));
    FILE *out = fopen(argv[2], "wb");
    if (!out) return 1;
    fwrite(&E0, sizeof(double), 1, out);
    fwrite(F, sizeof(double), 3 * (size_t)n, out);
    fwrite(H, sizeof(double), 3 * (size_t)n, out);
    const double B[3] = {0.0, 0.0, 0.5};
    CHECK(sl_step(sys, 10, 1.0, 300.0, B));
    uint64_t step = 0;
    CHECK(sl_get_state(sys, pos, vel, spins, NULL, NULL, NULL, &step));
    CHECK(sl_energy_forces_fields(sys, &E1, NULL, NULL, NULL));
    fwrite(pos, sizeof(double), 3 * (size_t)n, out);
    fwrite(spins, sizeof(double), 3 * (size_t)n, out);
    fwrite(&E1, sizeof(double), 1, out);
    int64_t st = (int64_t)step;
    fwrite(&st, sizeof(int64_t), 1, out);
    fclose(out);
    sl_destroy_system(sys);
    return 0;
}
