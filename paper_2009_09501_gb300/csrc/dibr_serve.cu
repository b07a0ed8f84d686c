// dibr_serve.cu -- serving loop: concurrent streams with continuous batching.
#include "dibr.h"
#include "dibr_context.h"

void dibr_ctx::shutdown_serving() {}

extern "C" {

dibr_status dibr_open_stream(dibr_ctx *c, int, int, const dibr_params *, int *) {
  if (c) c->set_error("serving loop not built yet");
  return DIBR_E_INVALID;
}
dibr_status dibr_submit_frame(dibr_ctx *c, int, uint64_t, const dibr_image *, const dibr_outputs *) {
  if (c) c->set_error("serving loop not built yet");
  return DIBR_E_CLOSED;
}
dibr_status dibr_poll(dibr_ctx *c, dibr_completion *, int, int *n_out, int) {
  if (n_out) *n_out = 0;
  return c ? DIBR_NOT_READY : DIBR_E_INVALID;
}
dibr_status dibr_close_stream(dibr_ctx *c, int) { return c ? DIBR_E_CLOSED : DIBR_E_INVALID; }

}  // extern "C"
