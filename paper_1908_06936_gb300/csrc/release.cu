// release_extra: frees the device buffers, the look-ahead stream and its events held by the
// mixed-precision, gradient, prediction, Fisher and batched paths of a context.
#include "ctx.cuh"

namespace exa {
void release_extra(exa_ctx* c) {
  DevBuf* bufs[] = {&c->mx_sigma, &c->mx_split, &c->mx_split2, &c->mx_split3, &c->mx_split4, &c->mx_split_b, &c->mx_vec, &c->mx_w2, &c->mx_wall, &c->mx_dscr, &c->mx_offmax, &c->mx_symv, &c->gr_part, &c->gr_xsplit, &c->gr_lsplit, &c->gr_t, &c->gr_blocks, &c->pr_c, &c->pr_y, &c->fs_m,
                    &c->bt_mat, &c->bt_meta, &c->bt_vec, &c->bt_work, &c->bt_mat2, &c->bt_tasks, &c->bt_ps, &c->bt_ws};
  for (DevBuf* b : bufs) {
    if (b->p) cudaFree(b->p);
    c->held_bytes -= b->bytes;
    b->p = nullptr;
    b->bytes = 0;
  }
  if (c->side) cudaStreamDestroy(c->side);
  c->side = nullptr;
  for (int i = 0; i < 2; ++i)
    if (c->la_ev[i]) cudaEventDestroy(c->la_ev[i]);
}
}  // namespace exa


