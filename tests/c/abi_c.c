/* The C ABI used from plain C (no Python, no torch): argument checks and the
 * memory contract without a GPU ("host"), then a short run with caller-owned
 * device memory and a checkpoint round trip ("gpu", with the checkpoint path).
 * Exit status 0 on success; each failed check prints a
 * line and makes it 1. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "tlbm.h"

static int failures = 0;
#define CHECK(cond, ...)                                   \
    do {                                                   \
        if (!(cond)) {                                     \
            fprintf(stderr, "FAIL %s:%d: ", __FILE__, __LINE__); \
            fprintf(stderr, __VA_ARGS__);                  \
            fprintf(stderr, "\n");                         \
            ++failures;                                    \
        }                                                  \
    } while (0)

static int host_checks(void) {
    tlbm_t h = NULL;
    /* invalid arguments come back as codes, with a message and a NULL handle */
    CHECK(tlbm_create(&h, 2, 10, 1, TLBM_D2Q9_D2Q5, 1e5, 0.71, 0.1, TLBM_FP32, NULL) == TLBM_ERR_ARG, "nx = 2");
    CHECK(h == NULL, "handle after a failed create");
    CHECK(strlen(tlbm_last_error(NULL)) > 0, "error text");
    CHECK(tlbm_create(&h, 10, 10, 1, TLBM_D2Q9_D2Q5, -1.0, 0.71, 0.1, TLBM_FP32, NULL) == TLBM_ERR_ARG, "Ra < 0");
    CHECK(tlbm_create(&h, 10, 10, 1, TLBM_D2Q9_D2Q5, 1e5, 0.71, 0.1, 9, NULL) == TLBM_ERR_UNSUPPORTED, "precision");
    tlbm_params p;
    tlbm_default_params(&p);
    CHECK(p.walls == TLBM_RB && p.streaming == TLBM_STREAM_PULL && isnan(p.nu), "defaults");
    /* the in-place scheme needs one population buffer less */
    size_t b2 = 0, b1 = 0;
    CHECK(tlbm_create(&h, 257, 129, 1, TLBM_D2Q9_D2Q5, 1e6, 0.71, 0.1, TLBM_FP32, &p) == TLBM_OK, "create");
    CHECK(tlbm_required_bytes(h, &b2) == TLBM_OK && b2 % 256 == 0, "required bytes");
    CHECK(tlbm_step(h, 1) == TLBM_ERR_UNBOUND, "step before bind");
    tlbm_destroy(h);
    p.streaming = TLBM_STREAM_INPLACE;
    CHECK(tlbm_create(&h, 257, 129, 1, TLBM_D2Q9_D2Q5, 1e6, 0.71, 0.1, TLBM_FP32, &p) == TLBM_OK, "create");
    CHECK(tlbm_required_bytes(h, &b1) == TLBM_OK, "required bytes");
    tlbm_destroy(h);
    CHECK(b2 - b1 >= (size_t)14 * 4 * 257 * 129, "in place saves a population buffer (%zu vs %zu)", b1, b2);
    return failures;
}

/* one cell, caller-owned device memory; returns the Nusselt number */
static double run(int streaming, int steps, double* mass0, double* mass1) {
    tlbm_params p;
    tlbm_default_params(&p);
    p.streaming = streaming;
    tlbm_t h = NULL;
    CHECK(tlbm_create(&h, 65, 33, 1, TLBM_D2Q9_D2Q5, 1e5, 0.71, 0.1, TLBM_FP64, &p) == TLBM_OK, "create");
    size_t bytes = 0;
    tlbm_required_bytes(h, &bytes);
    void* mem = NULL;
    CHECK(cudaMalloc(&mem, bytes) == cudaSuccess, "cudaMalloc");
    CHECK(tlbm_bind_memory(h, mem, bytes) == TLBM_OK, "bind: %s", tlbm_last_error(h));
    CHECK(tlbm_init(h, 1, 1e-3) == TLBM_OK, "init");
    double ek = 0.0;
    CHECK(tlbm_energy(h, &ek, mass0) == TLBM_OK, "energy");
    CHECK(tlbm_step(h, steps) == TLBM_OK, "step: %s", tlbm_last_error(h));
    double nu = 0.0;
    CHECK(tlbm_nusselt(h, &nu) == TLBM_OK, "nusselt");
    CHECK(tlbm_energy(h, &ek, mass1) == TLBM_OK, "energy");
    int div = 1;
    int64_t t = 0;
    CHECK(tlbm_status(h, &div, &t) == TLBM_OK && !div && t == steps, "status");
    /* the canonical populations come back in host memory */
    const size_t n = (size_t)65 * 33;
    double* f = (double*)malloc(9 * n * sizeof(double));
    double* g = (double*)malloc(5 * n * sizeof(double));
    CHECK(tlbm_get_populations(h, f, g) == TLBM_OK, "get populations");
    double rho = 0.0;
    for (size_t k = 0; k < 9 * n; ++k) rho += f[k];
    CHECK(fabs(rho - *mass1) < 1e-9 * *mass1, "sum of host populations %.17g vs mass %.17g", rho, *mass1);
    free(f);
    free(g);
    tlbm_destroy(h);
    cudaFree(mem);
    return nu;
}

/* checkpoint round trip: save after 40 steps, step on; a second handle loads
 * the file and steps on as well; the states must agree bit for bit */
static void checkpoint_check(const char* path) {
    tlbm_t h[2] = {NULL, NULL};
    void* mem[2] = {NULL, NULL};
    size_t bytes = 0;
    for (int k = 0; k < 2; ++k) {
        CHECK(tlbm_create(&h[k], 48, 24, 1, TLBM_D2Q9_D2Q5, 1e5, 0.71, 0.1, TLBM_FP16_OFFSET, NULL) == TLBM_OK,
              "create");
        tlbm_required_bytes(h[k], &bytes);
        CHECK(cudaMalloc(&mem[k], bytes) == cudaSuccess, "cudaMalloc");
        CHECK(tlbm_bind_memory(h[k], mem[k], bytes) == TLBM_OK, "bind");
    }
    CHECK(tlbm_init(h[0], 9, 1e-3) == TLBM_OK, "init");
    CHECK(tlbm_step(h[0], 40) == TLBM_OK, "step");
    CHECK(tlbm_save(h[0], path) == TLBM_OK, "save: %s", tlbm_last_error(h[0]));
    CHECK(tlbm_step(h[0], 17) == TLBM_OK, "step");
    CHECK(tlbm_load(h[1], path) == TLBM_OK, "load: %s", tlbm_last_error(h[1]));
    int64_t t = 0;
    CHECK(tlbm_status(h[1], NULL, &t) == TLBM_OK && t == 40, "step counter after load");
    CHECK(tlbm_step(h[1], 17) == TLBM_OK, "step");
    const size_t n = (size_t)48 * 24;
    double* f[2];
    for (int k = 0; k < 2; ++k) {
        f[k] = (double*)malloc(9 * n * sizeof(double));
        CHECK(tlbm_get_populations(h[k], f[k], NULL) == TLBM_OK, "get populations");
    }
    CHECK(memcmp(f[0], f[1], 9 * n * sizeof(double)) == 0, "resumed state differs");
    for (int k = 0; k < 2; ++k) {
        free(f[k]);
        tlbm_destroy(h[k]);
        cudaFree(mem[k]);
    }
    remove(path);
}

static int gpu_checks(const char* path) {
    double m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    const double a = run(TLBM_STREAM_PULL, 301, &m0, &m1);
    const double b = run(TLBM_STREAM_INPLACE, 301, &m2, &m3);
    CHECK(fabs(m1 - m0) < 1e-12 * m0, "mass drift %.3e", fabs(m1 - m0) / m0);
    CHECK(a == b, "two-buffer and in-place Nusselt numbers differ: %.17g vs %.17g", a, b);
    CHECK(a > 0.99 && a < 5.0, "Nusselt number %g", a);
    printf("nusselt %.17g %.17g mass %.17g\n", a, b, m1);
    checkpoint_check(path);
    return failures;
}

int main(int argc, char** argv) {
    if (argc < 2) return 2;
    int rc = 0;
    if (!strcmp(argv[1], "host")) rc = host_checks();
    else if (!strcmp(argv[1], "gpu") && argc > 2) rc = host_checks() + gpu_checks(argv[2]);
    else return 2;
    printf("%s: %d failure(s)\n", argv[1], rc);
    return rc ? 1 : 0;
}
