/* A plain C client of the library's C ABI (include/pmf.h), built by the tests
 * with gcc and linked against libpmf.so: no Python, no torch.
 *
 *   abi_client host              host-only calls (sizes, statuses, strings)
 *   abi_client solve IN OUT      solve one instance read from IN through a
 *                                batch (pmf_create_batch ... pmf_get_cuts)
 *   abi_client noalloc IN OUT    the same instance through pmf_solve_noalloc
 *   abi_client server IN OUT     the same instance through a running server
 *                                kernel (pmf_server_create ... pmf_server_read),
 *                                loaded twice: into its own slot and into a
 *                                second slot that uses the first one's image
 *
 * IN (little-endian int32): H, W, n_lambda, lambdas[n_lambda], then H*W each
 * of w_h, w_v, src0, slope, sink.  OUT: n_lambda int64 flows, then
 * n_lambda*H*W uint8 masks.  Exit status 0 on success. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "pmf.h"

#define CHECK(x)                                                                 \
    do {                                                                         \
        pmf_status s_ = (x);                                                     \
        if (s_ != PMF_OK) {                                                      \
            fprintf(stderr, "%s:%d %s -> %s (%s)\n", __FILE__, __LINE__, #x,     \
                    pmf_status_string(s_), pmf_last_error());                    \
            return 1;                                                            \
        }                                                                        \
    } while (0)

static int host_calls(void) {
    if (!pmf_version() || !pmf_version()[0]) return 2;
    for (int s = PMF_OK; s <= PMF_ERR_NOT_READY; ++s)
        if (!pmf_status_string((pmf_status)s)) return 3;
    int32_t h[2] = {64, 240}, w[2] = {64, 320}, im[3] = {0, 1, 1};
    pmf_batch_desc d = {2, h, w, 3, im, 20, 0};
    size_t bytes = 0;
    CHECK(pmf_workspace_size(&d, &bytes));
    if (bytes == 0) return 4;
    size_t bytes2 = 0;
    d.max_lambdas = 40;
    CHECK(pmf_workspace_size(&d, &bytes2));
    if (bytes2 <= bytes) return 5;                     /* more lambdas, more mask bytes */
    if (pmf_workspace_size(NULL, &bytes) != PMF_ERR_INVALID_ARG) return 6;
    h[0] = 0;
    if (pmf_workspace_size(&d, &bytes) != PMF_ERR_INVALID_ARG) return 7;
    if (pmf_sync(NULL, NULL) != PMF_ERR_INVALID_ARG) return 8;
    pmf_destroy_batch(NULL);
    printf("host ok %zu %zu\n", bytes, bytes2);
    return 0;
}

typedef struct {
    int32_t H, W, m;
    int32_t *lam, *arr;   /* lambdas[m]; w_h, w_v, src0, slope, sink, H*W each */
} problem;

static int read_problem(const char *path, problem *p) {
    FILE *f = fopen(path, "rb");
    if (!f) return 10;
    int32_t hdr[3];
    if (fread(hdr, 4, 3, f) != 3 || hdr[0] < 1 || hdr[1] < 1 || hdr[2] < 1) { fclose(f); return 11; }
    p->H = hdr[0]; p->W = hdr[1]; p->m = hdr[2];
    const size_t n = (size_t)p->H * p->W;
    p->lam = malloc(4 * (size_t)p->m);
    p->arr = malloc(4 * 5 * n);
    if (!p->lam || !p->arr) { fclose(f); return 12; }
    if (fread(p->lam, 4, p->m, f) != (size_t)p->m || fread(p->arr, 4, 5 * n, f) != 5 * n) { fclose(f); return 13; }
    fclose(f);
    return 0;
}

static int write_result(const char *path, const int64_t *flows, const uint8_t *masks, int32_t m, size_t n) {
    FILE *o = fopen(path, "wb");
    if (!o) return 19;
    const int ok = fwrite(flows, 8, m, o) == (size_t)m && fwrite(masks, 1, n * (size_t)m, o) == n * (size_t)m;
    fclose(o);
    return ok ? 0 : 20;
}

static int solve(const char *in_path, const char *out_path) {
    problem p;
    int rc = read_problem(in_path, &p);
    if (rc) return rc;
    const int32_t H = p.H, W = p.W, m = p.m;
    const size_t n = (size_t)H * W;
    int32_t *lam = p.lam, *arr = p.arr;
    int32_t im0 = 0;
    pmf_batch_desc d = {1, &H, &W, 1, &im0, m, 0};
    size_t bytes = 0;
    CHECK(pmf_workspace_size(&d, &bytes));
    void *ws = NULL;
    if (cudaMalloc(&ws, bytes) != cudaSuccess) return 14;
    pmf_batch *b = NULL;
    CHECK(pmf_create_batch(&d, ws, bytes, NULL, &b));
    CHECK(pmf_set_capacities(b, 0, arr, arr + n, 0));
    CHECK(pmf_set_terminals(b, 0, arr + 2 * n, arr + 3 * n, arr + 4 * n, 0));
    CHECK(pmf_solve_schedule(b, lam, m, NULL));
    /* wait for the instance through pmf_poll, then read it before pmf_sync */
    for (long spin = 0;; ++spin) {
        uint8_t done = 0;
        int32_t n_done = 0;
        CHECK(pmf_poll(b, &done, &n_done));
        if (done && n_done == 1) break;
        if (spin > 100000000L) return 21;
    }
    int64_t f_early = 0;
    CHECK(pmf_get_flow(b, 0, m - 1, &f_early));
    pmf_status per = PMF_OK;
    CHECK(pmf_sync(b, &per));
    if (per != PMF_OK) return 15;
    int64_t *flows = malloc(8 * (size_t)m);
    uint8_t *masks = malloc(n * (size_t)m);
    if (!flows || !masks) return 16;
    CHECK(pmf_get_flows(b, 0, flows));
    CHECK(pmf_get_cuts(b, 0, masks, 0));
    /* one value and one cut through the single-result calls as well */
    int64_t f_last = 0;
    CHECK(pmf_get_flow(b, 0, m - 1, &f_last));
    if (f_last != flows[m - 1] || f_early != f_last) return 17;
    uint8_t *one = malloc(n);
    CHECK(pmf_get_cut(b, 0, m - 1, one, 0));
    if (memcmp(one, masks + (size_t)(m - 1) * n, n) != 0) return 18;
    pmf_destroy_batch(b);
    cudaFree(ws);
    rc = write_result(out_path, flows, masks, m, n);
    free(lam); free(arr); free(flows); free(masks); free(one);
    if (!rc) printf("solve ok\n");
    return rc;
}

static int solve_noalloc(const char *in_path, const char *out_path) {
    problem p;
    int rc = read_problem(in_path, &p);
    if (rc) return rc;
    const size_t n = (size_t)p.H * p.W;
    int32_t *d_arr = NULL;
    uint8_t *d_masks = NULL;
    if (cudaMalloc((void **)&d_arr, 4 * 5 * n) != cudaSuccess) return 30;
    if (cudaMalloc((void **)&d_masks, n * (size_t)p.m) != cudaSuccess) return 31;
    if (cudaMemcpy(d_arr, p.arr, 4 * 5 * n, cudaMemcpyHostToDevice) != cudaSuccess) return 32;
    int64_t *flows = malloc(8 * (size_t)p.m);
    uint8_t *masks = malloc(n * (size_t)p.m);
    if (!flows || !masks) return 33;
    CHECK(pmf_solve_noalloc(p.H, p.W, d_arr, d_arr + n, d_arr + 2 * n, d_arr + 3 * n, d_arr + 4 * n,
                            p.lam, p.m, d_masks, flows, NULL));
    if (cudaMemcpy(masks, d_masks, n * (size_t)p.m, cudaMemcpyDeviceToHost) != cudaSuccess) return 34;
    cudaFree(d_arr);
    cudaFree(d_masks);
    rc = write_result(out_path, flows, masks, p.m, n);
    free(p.lam); free(p.arr); free(flows); free(masks);
    if (!rc) printf("noalloc ok\n");
    return rc;
}

static int solve_server(const char *in_path, const char *out_path) {
    problem p;
    int rc = read_problem(in_path, &p);
    if (rc) return rc;
    const size_t n = (size_t)p.H * p.W;
    pmf_server_desc d = {3, p.H, p.W, p.m, 0};
    size_t bytes = 0;
    CHECK(pmf_server_workspace_size(&d, &bytes));
    void *ws = NULL;
    if (cudaMalloc(&ws, bytes) != cudaSuccess) return 40;
    pmf_server *s = NULL;
    CHECK(pmf_server_create(&d, ws, bytes, &s));
    CHECK(pmf_server_start(s, 60.0));
    const int32_t *a = p.arr;
    CHECK(pmf_server_load(s, 2, 2, p.H, p.W, a, a + n, a + 2 * n, a + 3 * n, a + 4 * n, p.lam, p.m));
    CHECK(pmf_server_load(s, 0, 2, p.H, p.W, NULL, NULL, a + 2 * n, a + 3 * n, a + 4 * n, p.lam, p.m));
    const int32_t slots[2] = {2, 0};
    CHECK(pmf_server_post(s, slots, 2));
    for (long spin = 0;; ++spin) {
        uint8_t done[3] = {0, 0, 0};
        int32_t n_done = 0;
        CHECK(pmf_server_poll(s, done, &n_done));
        if (done[0] && done[2] && n_done == 2) break;
        if (spin > 200000000L) return 41;
    }
    int64_t *flows = malloc(8 * (size_t)p.m), *flows2 = malloc(8 * (size_t)p.m);
    uint8_t *masks = malloc(n * (size_t)p.m), *masks2 = malloc(n * (size_t)p.m);
    if (!flows || !flows2 || !masks || !masks2) return 42;
    CHECK(pmf_server_read(s, 0, masks, flows));
    CHECK(pmf_server_read(s, 2, masks2, flows2));
    if (memcmp(flows, flows2, 8 * (size_t)p.m) != 0 || memcmp(masks, masks2, n * (size_t)p.m) != 0) return 43;
    if (pmf_server_read(s, 2, masks2, flows2) != PMF_ERR_NOT_READY) return 44;   /* read once */
    CHECK(pmf_server_stop(s));
    pmf_server_destroy(s);
    cudaFree(ws);
    rc = write_result(out_path, flows, masks, p.m, n);
    free(p.lam); free(p.arr); free(flows); free(flows2); free(masks); free(masks2);
    if (!rc) printf("server ok\n");
    return rc;
}

int main(int argc, char **argv) {
    if (argc >= 2 && strcmp(argv[1], "host") == 0) return host_calls();
    if (argc >= 4 && strcmp(argv[1], "solve") == 0) return solve(argv[2], argv[3]);
    if (argc >= 4 && strcmp(argv[1], "noalloc") == 0) return solve_noalloc(argv[2], argv[3]);
    if (argc >= 4 && strcmp(argv[1], "server") == 0) return solve_server(argv[2], argv[3]);
    fprintf(stderr, "usage: abi_client host | solve IN OUT | noalloc IN OUT | server IN OUT\n");
    return 64;
}
