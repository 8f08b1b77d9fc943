/* A plain C client of libgcp: no Python, no torch.  Solves a diagonal
 * Hamiltonian, whose ground-state density matrix is known in closed form
 * (the projector on the N lowest diagonal entries), in FP64 and in the
 * split-precision mixed mode, through gcp_create / gcp_solve / gcp_destroy,
 * and checks D, Tr D and E.  Exit status 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "gcp.h"

static int check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
    return 1;
  }
  return 0;
}

static int cmp_double(const void* a, const void* b) {
  const double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

static int run(void* h, const double* Hh, double* Dh, double* dH, double* dD, int M, int N,
               int prec, double tol, double dtol) {
  gcp_options o;
  gcp_result r;
  gcp_default_options(&o);
  o.prec = prec;
  o.tol = tol;
  gcp_status st = gcp_solve(h, dH, M, N, M, GCP_F64, dD, M, GCP_F64, &r, &o);
  if (st != GCP_OK) {
    fprintf(stderr, "gcp_solve(prec %d): %s (%s)\n", prec, gcp_status_string(st),
            gcp_last_error(h));
    return 1;
  }
  if (check_cuda(cudaMemcpy(Dh, dD, sizeof(double) * M * M, cudaMemcpyDeviceToHost), "copy D"))
    return 1;
  /* the N lowest diagonal entries of H */
  double* d = (double*)malloc(sizeof(double) * M);
  for (int i = 0; i < M; ++i) d[i] = Hh[(size_t)i * M + i];
  qsort(d, M, sizeof(double), cmp_double);
  const double cut = 0.5 * (d[N - 1] + d[N]);
  double e_ref = 0.0, tr = 0.0, err = 0.0;
  for (int k = 0; k < N; ++k) e_ref += d[k];
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      const double want = (i == j && Hh[(size_t)i * M + i] < cut) ? 1.0 : 0.0;
      const double x = Dh[(size_t)i * M + j];
      if (fabs(x - want) > err) err = fabs(x - want);
      if (i == j) tr += x;
    }
  free(d);
  printf("prec %d: %d steps, max|D - D_ref| = %.2e, |Tr D - N| = %.2e, |E - E_ref| = %.2e\n",
         prec, r.iters, err, fabs(tr - N), fabs(r.energy - e_ref));
  return !(err <= dtol && fabs(tr - N) <= 1e-9 && fabs(r.energy - e_ref) <= 1e-9 * fabs(e_ref));
}

int main(void) {
  const int M = 300, N = 75;
  double* Hh = (double*)calloc((size_t)M * M, sizeof(double));
  double* Dh = (double*)malloc(sizeof(double) * M * M);
  /* diagonal entries: two bands [-1, -0.05] and [0.05, 1] in a scrambled
   * order (a fixed linear-congruential sequence) */
  unsigned long long s = 12345;
  for (int i = 0; i < M; ++i) {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    const double u = (double)(s >> 11) / 9007199254740992.0;
    const int occupied = ((i * 37) % M) < N;
    Hh[(size_t)i * M + i] = occupied ? -1.0 + 0.95 * u : 0.05 + 0.95 * u;
  }
  double *dH = NULL, *dD = NULL;
  if (check_cuda(cudaMalloc((void**)&dH, sizeof(double) * M * M), "cudaMalloc") ||
      check_cuda(cudaMalloc((void**)&dD, sizeof(double) * M * M), "cudaMalloc") ||
      check_cuda(cudaMemcpy(dH, Hh, sizeof(double) * M * M, cudaMemcpyHostToDevice), "copy H"))
    return 1;
  void* h = NULL;
  if (gcp_create(&h) != GCP_OK) return 1;
  int bad = run(h, Hh, Dh, dH, dD, M, N, GCP_FP64, 1e-12, 1e-10);
  bad |= run(h, Hh, Dh, dH, dD, M, N, GCP_MIXED_FP16, 1e-10, 1e-8);
  gcp_destroy(h);
  cudaFree(dH);
  cudaFree(dD);
  free(Hh);
  free(Dh);
  printf(bad ? "FAILED\n" : "ok\n");
  return bad;
}
