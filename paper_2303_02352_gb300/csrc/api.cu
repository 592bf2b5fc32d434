// Small C-ABI entry points of libamg: defaults, hierarchy queries, errors,
// teardown.  The paper's parameter file (App. A, Listing 1) maps onto
// amg_params; its defaults are the settings of the experiments of Sec. 5.
#include <cstring>
#include <string>

#include "amg_internal.cuh"

static thread_local std::string g_setup_error;

void amg_set_setup_error(const std::string& msg) { g_setup_error = msg; }

extern "C" void amg_params_default(amg_params* p) {
  if (!p) return;
  p->aggr_steps = 3;      // Listing 1 aggrsweeps = 2; Sec. 5: aggregates of size at most 8
  p->max_levels = 39;     // Listing 1
  p->coarse_size = 0;     // Sec. 5: 40 * nd
  p->pre_sweeps = 4;      // Sec. 5 / Listing 1
  p->post_sweeps = 4;
  p->coarse_sweeps = 20;  // Sec. 5 / Listing 1 relaxnumber_coarse
  p->precision = AMG_FP64;
  p->true_res_every = 50;
  p->use_graph = 1;
  p->graph_batch = 4;
  p->num_parts = 1;
  p->cycle = 0;
  p->relax_type = 4;
  p->prolong_scale = 0;
}

extern "C" amg_status amg_info(const amg_handle* h, amg_info_t* info) {
  if (!h || !info) return AMG_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  info->num_levels = h->nl;
  double tot = 0.0;
  for (int k = 0; k < h->nl && k < 40; ++k) {
    info->n[k] = h->L[k].n;
    info->nnz[k] = h->L[k].nnz;
    tot += (double)h->L[k].nnz;
  }
  info->opc = h->L[0].nnz ? tot / (double)h->L[0].nnz : 0.0;
  info->num_pairwise = h->npair;
  info->setup_ms = h->setup_ms;
  info->vcycle_bytes = h->bytes_vcycle;
  info->iteration_bytes = h->bytes_iter;
  info->vcycle_launches = h->launches_vcycle;
  info->iteration_launches = h->launches_iter;
  info->precision = h->p.precision;
  info->setup_match_ms = h->match_ms;
  info->setup_galerkin_ms = h->galerkin_ms;
  info->setup_spgemm_ms = h->spgemm_ms;
  info->last_solve_launches = h->launches_last_solve;
  info->bottom_level = h->kb < h->nl ? h->kb : h->nl;
  for (int k = 0; k < h->nl && k < 40; ++k) {
    const Level& L = h->L[k];
    info->tile_rows[k] = L.pipe ? L.R : 0;
    info->stage_scale[k] = L.pipe ? (L.sb == 5 ? 2 : (L.sb == 6 ? 1 : L.sb)) : 0;
    info->consumer_groups[k] = L.pipe ? ((L.sb == 5 || L.sb == 6) ? 2 : 1) : 0;
    info->column_patterns[k] = L.pat ? L.npat : 0;
    info->column_form[k] = L.pat;
  }
  info->outer_patterns = h->nl > 0 && h->L[0].patd ? h->L[0].npat : 0;
  info->outer_column_form = h->nl > 0 ? h->L[0].patd : 0;
  return AMG_OK;
}

extern "C" amg_status amg_get_aggregates(amg_handle* h, int32_t level, int32_t* agg_host) {
  if (!h || !agg_host) return AMG_ERR_INVALID_ARG;
  if (level < 0 || level >= h->nl - 1) return amg_fail(h, AMG_ERR_INVALID_ARG, "level %d has no aggregates", level);
  const Level& L = h->L[level];
  AMG_CK(h, cudaMemcpyAsync(agg_host, L.agg, sizeof(int32_t) * (size_t)L.n, cudaMemcpyDeviceToHost, h->stream));
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

extern "C" amg_status amg_get_level_csr(amg_handle* h, int32_t level, int32_t* rp, int32_t* ci, double* v) {
  if (!h || !rp || !ci || !v) return AMG_ERR_INVALID_ARG;
  if (level < 0 || level >= h->nl) return amg_fail(h, AMG_ERR_INVALID_ARG, "bad level %d", level);
  const Level& L = h->L[level];
  AMG_CK(h, cudaMemcpyAsync(rp, L.rp, sizeof(int32_t) * (size_t)(L.n + 1), cudaMemcpyDeviceToHost, h->stream));
  AMG_CK(h, cudaMemcpyAsync(ci, L.ci, sizeof(int32_t) * (size_t)L.nnz, cudaMemcpyDeviceToHost, h->stream));
  AMG_CK(h, cudaMemcpyAsync(v, L.v, sizeof(double) * (size_t)L.nnz, cudaMemcpyDeviceToHost, h->stream));
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

extern "C" amg_status amg_get_l1(amg_handle* h, int32_t level, double* l1) {
  if (!h || !l1) return AMG_ERR_INVALID_ARG;
  if (level < 0 || level >= h->nl) return amg_fail(h, AMG_ERR_INVALID_ARG, "bad level %d", level);
  const Level& L = h->L[level];
  AMG_CK(h, cudaMemcpyAsync(l1, L.l1, sizeof(double) * (size_t)L.n, cudaMemcpyDeviceToHost, h->stream));
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

extern "C" const char* amg_last_error(const amg_handle* h) {
  if (!h) return g_setup_error.c_str();
  return h->err.c_str();
}

void amg_release_graphs(amg_handle* h);

extern "C" void amg_destroy(amg_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  amg_release_graphs(h);
  amg_adj_destroy(h);
  amg_free_bottom(h);
  amg_free_all(h);
  delete h;
}
