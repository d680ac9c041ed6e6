/*
 * A plain C user of the library's C ABI (include/stp.h), for the GPU tests:
 * reads q and params of E elements from binary files, runs the STP through
 * the host-buffer entry point (no CUDA or Python in this program), writes the
 * average and the faces, and checks two argument errors on the way.
 *
 *   abi_host_predict ORDER DX DT E q.bin params.bin avg.bin faces.bin
 */
#include <stdio.h>
#include <stdlib.h>

#include "stp.h"

static int read_all(const char* path, double* buf, size_t n) {
  FILE* f = fopen(path, "rb");
  if (!f) return -1;
  const size_t got = fread(buf, sizeof(double), n, f);
  fclose(f);
  return got == n ? 0 : -1;
}

static int write_all(const char* path, const double* buf, size_t n) {
  FILE* f = fopen(path, "wb");
  if (!f) return -1;
  const size_t put = fwrite(buf, sizeof(double), n, f);
  fclose(f);
  return put == n ? 0 : -1;
}

int main(int argc, char** argv) {
  if (argc != 9) {
    fprintf(stderr, "usage: %s ORDER DX DT E q.bin params.bin avg.bin faces.bin\n", argv[0]);
    return 2;
  }
  const int order = atoi(argv[1]);
  const double dx = atof(argv[2]), dt = atof(argv[3]);
  const long long E = atoll(argv[4]);
  const size_t N = (size_t)order + 1, n3 = N * N * N;
  double* q = malloc(sizeof(double) * E * n3 * 9);
  double* params = malloc(sizeof(double) * E * n3 * 3);
  double* avg = malloc(sizeof(double) * E * n3 * 9);
  double* faces = malloc(sizeof(double) * E * 6 * N * N * 9);
  if (!q || !params || !avg || !faces) return 3;
  if (read_all(argv[5], q, E * n3 * 9) || read_all(argv[6], params, E * n3 * 3)) return 4;

  stp_handle h = NULL;
  /* argument errors come back as statuses, before anything runs */
  if (stp_create(order, 8, dx, dt, &h) != STP_ERR_UNSUPPORTED || h != NULL) return 5;
  if (stp_create(order, 9, -dx, dt, &h) != STP_ERR_INVALID_ARG) return 6;
  stp_status s = stp_create(order, 9, dx, dt, &h);
  if (s != STP_OK) {
    fprintf(stderr, "stp_create: %s (%s)\n", stp_status_string(s), stp_last_error());
    return 7;
  }
  if (stp_nodes(h) != (int)N) return 8;
  s = stp_predict_host(h, E, q, params, avg, faces, NULL);
  if (s != STP_OK) {
    fprintf(stderr, "stp_predict_host: %s (%s)\n", stp_status_string(s), stp_last_error());
    return 9;
  }
  if (stp_destroy(h) != STP_OK || stp_destroy(NULL) != STP_OK) return 10;
  if (write_all(argv[7], avg, E * n3 * 9) || write_all(argv[8], faces, E * 6 * N * N * 9)) return 11;
  free(q);
  free(params);
  free(avg);
  free(faces);
  printf("ok\n");
  return 0;
}
