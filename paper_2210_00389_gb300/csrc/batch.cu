// Batched counting of many independent graphs (tc_count_batch).
// Preliminary form: one graph object per input, counted in turn on the
// caller's stream.
#include <vector>

#include "internal.cuh"

using namespace tc;

extern "C" int tc_count_batch(const tc_csr_view* graphs, int32_t ngraphs, int mode,
                              const tc_options* opt, void* cuda_stream, uint64_t* counts_out,
                              int* status_out) {
  (void)opt;
  if (ngraphs < 0 || (ngraphs > 0 && (!graphs || !counts_out)))
    return fail(TC_ERR_INVALID_ARG, "tc_count_batch: bad arguments");
  if (mode != TC_MODE_COVER && mode != TC_MODE_PLAIN)
    return fail(TC_ERR_INVALID_ARG, "tc_count_batch: unknown mode %d", mode);
  for (int32_t i = 0; i < ngraphs; ++i) {
    tc_graph* g = nullptr;
    int st = tc_graph_create(&graphs[i], 0, cuda_stream, &g);
    uint64_t c = 0;
    if (st == TC_OK) st = tc_count(g, mode, &c);
    tc_graph_destroy(g);
    counts_out[i] = st == TC_OK ? c : 0;
    if (status_out) status_out[i] = st;
    if (st != TC_OK && st != TC_ERR_INVALID_GRAPH) return st;
  }
  return TC_OK;
}
