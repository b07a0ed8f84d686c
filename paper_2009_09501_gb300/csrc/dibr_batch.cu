// dibr_batch.cu -- batched synthesis of images of uneven sizes.
#include <string>

#include "dibr.h"
#include "dibr_context.h"
#include "dibr_internal.h"

using namespace dibr;

void dibr_ctx::release_batch_buffers() {
  for (DevBuf *b : {&batch_desc, &batch_img, &batch_depth}) {
    dev_free(b->ptr);
    b->ptr = nullptr;
    b->bytes = 0;
  }
}

extern "C" {

dibr_status dibr_enqueue_batch(dibr_ctx *c, int n, const dibr_image *imgs, const dibr_params *p,
                               int n_params, const dibr_outputs *outs) {
  if (!c || n < 0 || (n > 0 && (!imgs || !p || !outs))) return DIBR_E_INVALID;
  if (n_params != 1 && n_params != n) return DIBR_E_INVALID;
  for (int i = 0; i < n; ++i) {
    dibr_status s = dibr_enqueue_image(c, &imgs[i], &p[n_params == 1 ? 0 : i], &outs[i]);
    if (s != DIBR_OK) return s;
  }
  return DIBR_OK;
}

dibr_status dibr_synthesize_batch(dibr_ctx *c, int n, const dibr_image *imgs, const dibr_params *p,
                                  int n_params, const dibr_outputs *outs) {
  if (!c || n < 0 || (n > 0 && (!imgs || !p || !outs))) return DIBR_E_INVALID;
  if (n_params != 1 && n_params != n) return DIBR_E_INVALID;
  for (int i = 0; i < n; ++i) {
    dibr_status s = dibr_synthesize_image(c, &imgs[i], &p[n_params == 1 ? 0 : i], &outs[i]);
    if (s != DIBR_OK) return s;
  }
  return DIBR_OK;
}

}  // extern "C"
