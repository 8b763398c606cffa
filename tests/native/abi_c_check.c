/* The C-ABI used from plain C99 (no C++, no CUDA headers): the header
 * compiles with -pedantic, the library links, and the calls that need no GPU
 * answer as the header documents.  Exit status 0 on success. */
#include <stdio.h>
#include <string.h>

#include "srtm.h"

static int failures = 0;

#define EXPECT(cond)                                          \
  do {                                                        \
    if (!(cond)) {                                            \
      fprintf(stderr, "line %d: failed: %s\n", __LINE__, #cond); \
      ++failures;                                             \
    }                                                         \
  } while (0)

int main(void) {
  srtm_problem p;
  srtm_output out;
  srtm_tuning t;
  char detail[256];
  memset(&p, 0, sizeof p);
  memset(&out, 0, sizeof out);

  EXPECT(srtm_smoother(NULL, SRTM_FP64, &out, NULL, NULL) == SRTM_ERR_ARG);
  p.nx = 9;
  p.ny = 1;
  p.ratio = 2;
  p.n_slow = 3;
  EXPECT(srtm_smoother(&p, SRTM_MIXED, &out, NULL, NULL) == SRTM_ERR_UNSUPPORTED);
  EXPECT(srtm_last_error_detail(detail, (int)sizeof detail) > 0 && strstr(detail, "nx=9") != NULL);
  p.nx = 4;
  p.ratio = 0;
  EXPECT(srtm_filter(&p, SRTM_FP64, &out, NULL) == SRTM_ERR_ARG);
  p.ratio = 2;
  EXPECT(srtm_smoother(&p, (srtm_precision)7, &out, NULL, NULL) == SRTM_ERR_ARG);
  EXPECT(srtm_smoother_batch(NULL, SRTM_MIXED, &out, NULL, NULL) == SRTM_ERR_ARG);
  EXPECT(srtm_selftest_wait(0, NULL) == SRTM_ERR_ARG);

  EXPECT(srtm_get_tuning(4, SRTM_MIXED, &t) == SRTM_OK);
  EXPECT(t.scan_groups >= 1 && t.scan_elems >= 1 && t.recover_threads % 32 == 0);
  t.recover_threads = 48; /* not a multiple of 32 */
  EXPECT(srtm_set_tuning(4, SRTM_MIXED, &t) == SRTM_ERR_ARG);

  EXPECT(srtm_launches_per_call(1, 0) == 4);
  EXPECT(srtm_launches_per_call(0, 1) == 4);
  EXPECT(SRTM_OK == 0 && SRTM_ERR_NOT_PSD == -2 && SRTM_ERR_SINGULAR == -3);

  if (failures == 0) printf("ok\n");
  return failures == 0 ? 0 : 1;
}
