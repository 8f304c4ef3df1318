/* A plain C user of libdfb.so: host buffers in, host buffers out, no CUDA
 * headers.  Reads a scene file, composites its frames with progressive
 * accumulation (BLEND_DEPTH), writes the RGBA8 frame and the normalised
 * accumulation.
 *
 * Scene file (little endian):
 *   int32 W, H, T, frames
 *   per frame: int32 n, then n tile ids (int32), n order keys (float32),
 *              n*T*T*4 RGBA (float32, premultiplied), n*T*T depths (float32)
 * Output file: W*H uint32 RGBA8, then W*H*4 float32 accumulation mean.
 * Exit status 0 on success; the first failing call is printed.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "dfb.h"

static int check(int st, const char* what) {
  if (st != DFB_OK) fprintf(stderr, "%s: %s (%d)\n", what, dfb_error_string(st), st);
  return st;
}

static void* read_all(FILE* f, size_t bytes) {
  void* p = malloc(bytes ? bytes : 1);
  if (p && bytes && fread(p, 1, bytes, f) != bytes) {
    free(p);
    return NULL;
  }
  return p;
}

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s scene.bin out.bin\n", argv[0]);
    return 2;
  }
  FILE* in = fopen(argv[1], "rb");
  if (!in) return 2;
  int32_t hdr[4];
  if (fread(hdr, sizeof hdr, 1, in) != 1) return 2;
  const int W = hdr[0], H = hdr[1], T = hdr[2], frames = hdr[3];
  dfb_handle h = NULL;
  if (check(dfb_create(W, H, T, DFB_BLEND_DEPTH, &h), "dfb_create")) return 1;
  for (int f = 0; f < frames; ++f) {
    int32_t n = 0;
    if (fread(&n, sizeof n, 1, in) != 1) return 2;
    const size_t px = (size_t)T * T;
    int32_t* ids = read_all(in, sizeof(int32_t) * n);
    float* keys = read_all(in, sizeof(float) * n);
    float* rgba = read_all(in, sizeof(float) * 4 * px * n);
    float* depth = read_all(in, sizeof(float) * px * n);
    if (!ids || !keys || !rgba || !depth) return 2;
    const void** rp = malloc(sizeof(void*) * (n ? n : 1));
    const float** dp = malloc(sizeof(float*) * (n ? n : 1));
    for (int i = 0; i < n; ++i) {
      rp[i] = rgba + 4 * px * i;
      dp[i] = depth + px * i;
    }
    if (check(dfb_begin_frame(h, f > 0), "dfb_begin_frame")) return 1;
    if (check(dfb_submit_tiles(h, n, ids, keys, rp, dp, NULL, DFB_PTR_HOST), "dfb_submit_tiles"))
      return 1;
    /* the host copies are done: the buffers may be reused right away */
    free(ids); free(keys); free(rgba); free(depth); free(rp); free(dp);
    if (check(dfb_end_frame(h, NULL), "dfb_end_frame")) return 1;
  }
  fclose(in);
  uint32_t* rgba8 = malloc(sizeof(uint32_t) * W * H);
  float* mean = malloc(sizeof(float) * 4 * W * H);
  if (check(dfb_read_rgba8(h, rgba8), "dfb_read_rgba8")) return 1;
  if (check(dfb_read_accum(h, mean), "dfb_read_accum")) return 1;
  dfb_frame_stats st;
  if (check(dfb_get_stats(h, &st), "dfb_get_stats")) return 1;
  FILE* out = fopen(argv[2], "wb");
  if (!out) return 2;
  fwrite(rgba8, sizeof(uint32_t), (size_t)W * H, out);
  fwrite(mean, sizeof(float), (size_t)4 * W * H, out);
  fclose(out);
  printf("frames %d accumulated %d fragments %lld\n", frames, st.accumulated,
         (long long)st.fragments);
  free(rgba8);
  free(mean);
  return check(dfb_destroy(h), "dfb_destroy") ? 1 : 0;
}
