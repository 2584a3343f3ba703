// The learned initial guess wired into a handle: stage-start hook and training-data
// helpers.  Included at the end of bgk_lib.cu after bgk_mlp.cuh.

namespace {

int guess_buffers(bgk_handle* h) {
  const int F = guess_features(h->hm.dim), nm = h->nm;
  int rc = BGK_OK;
  if (!h->gX) rc = dalloc(h->gX, sizeof(float) * (size_t)h->nnode * F);
  if (rc == BGK_OK && !h->gY) rc = dalloc(h->gY, sizeof(float) * (size_t)h->nnode * nm);
  if (rc == BGK_OK && !h->Uhist) rc = dalloc(h->Uhist, sizeof(double) * (size_t)h->nnode * nm);
  if (rc == BGK_OK && !h->have_hist) {
    rc = dalloc(h->have_hist, sizeof(int));
    if (rc == BGK_OK) CK(cudaMemsetAsync(h->have_hist, 0, sizeof(int), h->stream));
  }
  return rc;
}

// Features of the current moments U[it & 1] into gX, then U_hist <- U.
void guess_features_launch(bgk_handle* h) {
  const int c = h->hm.ncell;
  k_guess_features<<<(c + 127) / 128, 128, 0, h->stream>>>(h->hm.dim, h->hm.ndof, h->hm.quad ? 1 : 0, c, h->geo,
                                                          h->hm.geo_stride,
                                                           h->U[0], h->U[1], h->ds, h->Uhist, h->have_hist, h->dt,
                                                           h->phys.nu, h->gX);
  k_guess_history<<<148 * 4, 256, 0, h->stream>>>(h->nnode, h->nm, h->U[0], h->U[1], h->ds, h->Uhist, h->have_hist);
}

// Stage start with a network attached: features -> BF16 network -> guessed moments
// (previous change + network correction) replace iterate 0's moments node by node
// (non-physical predictions are skipped).
int guess_hook(bgk_handle* h) {
  bgk_mlp* m = h->guess;
  guess_features_launch(h);
  mlp_forward<__nv_bfloat16>(m, h->stream, h->gX, h->nnode, m->pb);
  k_denorm<<<(int)(((int64_t)h->nnode * m->O + 255) / 256), 256, 0, h->stream>>>(
      m->act[3], h->nnode, m->O, m->norm + 2 * m->F, m->norm + 2 * m->F + m->O, h->gY);
  k_guess_apply<<<(h->nnode + 127) / 128, 128, 0, h->stream>>>(h->nnode, h->hm.dim, h->gY, h->gX, h->U[0], h->U[1],
                                                               h->ds);
  return cudaGetLastError() == cudaSuccess ? BGK_OK : BGK_E_CUDA;
}

}  // namespace

extern "C" {

int bgk_guess_dims(const bgk_handle* h, int* n_features, int* n_outputs) {
  if (!h) return BGK_E_INVALID;
  if (n_features) *n_features = guess_features(h->hm.dim);
  if (n_outputs) *n_outputs = h->nm;
  return BGK_OK;
}

int bgk_guess_features(bgk_handle* h, float* d_X) {
  if (!h || !d_X) return BGK_E_INVALID;
  int rc = guess_buffers(h);
  if (rc != BGK_OK) return rc;
  k_reset_state<<<1, 1, 0, h->stream>>>(h->ds);
  moments(h, 0);
  guess_features_launch(h);
  const size_t bytes = sizeof(float) * (size_t)h->nnode * guess_features(h->hm.dim);
  CK(cudaMemcpyAsync(d_X, h->gX, bytes, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return BGK_OK;
}

int bgk_guess_targets(bgk_handle* h, const double* d_Ustart, const float* d_X, float* d_Y) {
  if (!h || !d_Ustart || !d_X || !d_Y) return BGK_E_INVALID;
  k_reset_state<<<1, 1, 0, h->stream>>>(h->ds);
  moments(h, 0);
  k_guess_targets<<<(h->nnode + 127) / 128, 128, 0, h->stream>>>(h->nnode, h->hm.dim, d_Ustart, h->U[0], h->U[1],
                                                                 h->ds, d_X, d_Y);
  CK(cudaStreamSynchronize(h->stream));
  return BGK_OK;
}

int bgk_set_guess(bgk_handle* h, bgk_mlp* m) {
  if (!h) return BGK_E_INVALID;
  if (m && (m->F != guess_features(h->hm.dim) || m->O != h->nm)) return BGK_E_INVALID;
  CK(cudaStreamSynchronize(h->stream));
  if (m) {
    int rc = guess_buffers(h);
    if (rc == BGK_OK) rc = mlp_reserve(m, h->nnode);
    if (rc != BGK_OK) return rc;
    k_to_bf16<<<(m->np + 255) / 256, 256, 0, h->stream>>>(m->np, m->p, m->pb);
    m->pb_valid = true;
    CK(cudaStreamSynchronize(h->stream));
  }
  h->guess = m;
  // the step graphs change shape: capture them again
  int rc = recapture_steps(h);
  if (rc != BGK_OK) return rc;
  return BGK_OK;
}

}  // extern "C"
