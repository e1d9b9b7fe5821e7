/* A plain C consumer of the library's C ABI (include/elses.h), with no Python or torch: it reads
 * a system from a binary file, runs one energy + force evaluation on the current CUDA device and
 * writes the results to a binary file.
 *
 *   input : int n; double box[3]; elses_sk sk; elses_params params; double pos[n][3]
 *   output: double mu, e_band, f_free; double forces[n][3]
 *
 * Usage: energy_force <input> <output>. Exit status 0 on success, else 1 with a message.     */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "elses.h"

static int read_all(FILE* f, void* p, size_t bytes) { return fread(p, 1, bytes, f) == bytes; }

int main(int argc, char** argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s <input> <output>\n", argv[0]);
        return 1;
    }
    FILE* in = fopen(argv[1], "rb");
    if (!in) { fprintf(stderr, "cannot open %s\n", argv[1]); return 1; }
    int n = 0;
    double box[3];
    elses_sk sk;
    elses_params params;
    if (!read_all(in, &n, sizeof n) || n <= 0 || !read_all(in, box, sizeof box) ||
        !read_all(in, &sk, sizeof sk) || !read_all(in, &params, sizeof params)) {
        fprintf(stderr, "bad input header\n");
        fclose(in);
        return 1;
    }
    double* pos = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* forces = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    if (!pos || !forces || !read_all(in, pos, sizeof(double) * 3 * (size_t)n)) {
        fprintf(stderr, "bad input positions\n");
        fclose(in);
        return 1;
    }
    fclose(in);

    double *pos_dev = NULL, *forces_dev = NULL;
    if (cudaMalloc((void**)&pos_dev, sizeof(double) * 3 * (size_t)n) != cudaSuccess ||
        cudaMalloc((void**)&forces_dev, sizeof(double) * 3 * (size_t)n) != cudaSuccess) {
        fprintf(stderr, "device allocation failed\n");
        return 1;
    }
    cudaMemcpy(pos_dev, pos, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice);

    elses_system sys = NULL;
    double mu = 0.0, e_band = 0.0, f_free = 0.0;
    int rc = elses_build_clusters(&sys, n, pos_dev, box, &sk, &params, NULL);
    if (rc >= 0) rc = elses_energy_force(sys, &mu, &e_band, &f_free, forces_dev, NULL);
    if (rc < 0) {
        fprintf(stderr, "elses error %d: %s\n", rc, elses_last_error());
        elses_system_destroy(sys);
        return 1;
    }
    cudaMemcpy(forces, forces_dev, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost);
    elses_system_destroy(sys);
    cudaFree(pos_dev);
    cudaFree(forces_dev);

    FILE* out = fopen(argv[2], "wb");
    if (!out) { fprintf(stderr, "cannot open %s\n", argv[2]); return 1; }
    fwrite(&mu, sizeof mu, 1, out);
    fwrite(&e_band, sizeof e_band, 1, out);
    fwrite(&f_free, sizeof f_free, 1, out);
    fwrite(forces, sizeof(double), 3 * (size_t)n, out);
    fclose(out);
    free(pos);
    free(forces);
    return 0;
}
