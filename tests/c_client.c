/* A plain C client of libsfd (no Python, no torch): synthesizes a plucked,
 * a hammered and a bowed string, one of them read on the longitudinal
 * channel, alone and as one batch with host output, and writes every
 * string's samples as raw float32 to the file named by argv[1].
 * Used by tests/test_gpu_c_client.py, which compares them with the Python
 * binding's. */
#include <stdio.h>
#include <stdlib.h>

#include "sfd.h"

#define N 4000
#define CHECK(call)                                                            \
  do {                                                                         \
    sfd_status rc_ = (call);                                                   \
    if (rc_ != SFD_OK) {                                                       \
      fprintf(stderr, "%s failed: %d (%s)\n", #call, rc_, sfd_last_error());   \
      return 1;                                                                \
    }                                                                          \
  } while (0)

static int make(sfd_ctx* ctx, int which, sfd_string** s) {
  sfd_string_params p;
  sfd_params_default(&p);
  p.f0 = 110.0 + 40.0 * which;
  p.alpha = 3.0;
  if (which == 2) p.output = SFD_OUTPUT_LONGITUDINAL;
  CHECK(sfd_string_create(ctx, &p, s));
  if (which == 0) CHECK(sfd_excite_pluck(*s, 1e-3, 0.3));
  if (which == 1) CHECK(sfd_excite_hammer(*s, 6e-3, 3.0, 0.31, 3000.0, 2.5));
  if (which == 2) CHECK(sfd_excite_bow(*s, 0.2, 1.0, 0.17, 100.0, 0.1, -1.0));
  return 0;
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  sfd_ctx* ctx = NULL;
  CHECK(sfd_ctx_create(0, NULL, 64u << 20, &ctx));
  float* alone = malloc(sizeof(float) * 3 * N);
  float* batch = malloc(sizeof(float) * 3 * N);
  if (!alone || !batch) return 3;
  for (int w = 0; w < 3; ++w) {
    sfd_string* s = NULL;
    if (make(ctx, w, &s)) return 1;
    CHECK(sfd_synthesize(s, N / 2, alone + w * N, 0));            /* two calls continue the note */
    CHECK(sfd_synthesize(s, N - N / 2, alone + w * N + N / 2, 0));
    CHECK(sfd_string_destroy(s));
  }
  sfd_string* ss[3];
  for (int w = 0; w < 3; ++w)
    if (make(ctx, w, &ss[w])) return 1;
  sfd_batch* b = NULL;
  CHECK(sfd_batch_create(ctx, 3, ss, &b));
  int64_t ns[3] = {N, N, N}, offs[3] = {0, N, 2 * N};
  int32_t st[3] = {0, 0, 0};
  CHECK(sfd_batch_synthesize_host(b, ns, batch, offs, st));
  CHECK(sfd_batch_destroy(b));
  for (int w = 0; w < 3; ++w) CHECK(sfd_string_destroy(ss[w]));
  sfd_ctx_destroy(ctx);
  FILE* f = fopen(argv[1], "wb");
  if (!f) return 4;
  fwrite(alone, sizeof(float), 3 * N, f);
  fwrite(batch, sizeof(float), 3 * N, f);
  fclose(f);
  free(alone);
  free(batch);
  printf("ok\n");
  return 0;
}
