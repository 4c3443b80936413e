// Mixed-precision echo path, variant 0 (linear surface, analytic patterns), and
// the run-time dispatch to the variant launchers (see echo_mixed.cuh).
#define HARM_MIXED_VARIANT 0
#include "echo_mixed.cuh"

namespace harm {

cudaError_t mixed_generate_v1(const DevScene &, const MixedTables &, cudaStream_t, int, int, float *);
cudaError_t mixed_generate_v2(const DevScene &, const MixedTables &, cudaStream_t, int, int, float *);
cudaError_t mixed_generate_v3(const DevScene &, const MixedTables &, cudaStream_t, int, int, float *);
cudaError_t mixed_accumulate_v1(const DevScene &, const MixedTables &, cudaStream_t, int, int, void *, harm_dtype);
cudaError_t mixed_accumulate_v2(const DevScene &, const MixedTables &, cudaStream_t, int, int, void *, harm_dtype);
cudaError_t mixed_accumulate_v3(const DevScene &, const MixedTables &, cudaStream_t, int, int, void *, harm_dtype);
cudaError_t mixed_adjoint_v1(const DevScene &, const MixedTables &, cudaStream_t, int, int, const void *, harm_dtype,
                             double *, double *);
cudaError_t mixed_adjoint_v2(const DevScene &, const MixedTables &, cudaStream_t, int, int, const void *, harm_dtype,
                             double *, double *);
cudaError_t mixed_adjoint_v3(const DevScene &, const MixedTables &, cudaStream_t, int, int, const void *, harm_dtype,
                             double *, double *);
cudaError_t mixed_probe_v1(const DevScene &, const MixedTables &, cudaStream_t, int, int, int *, void *, void *, int *);
cudaError_t mixed_probe_v2(const DevScene &, const MixedTables &, cudaStream_t, int, int, int *, void *, void *, int *);
cudaError_t mixed_probe_v3(const DevScene &, const MixedTables &, cudaStream_t, int, int, int *, void *, void *, int *);
cudaError_t mixed_batch_v1(const BatchLaunch &, cudaStream_t);
cudaError_t mixed_batch_v2(const BatchLaunch &, cudaStream_t);
cudaError_t mixed_batch_v3(const BatchLaunch &, cudaStream_t);

static_assert(sizeof(MixedArgs) <= 2048, "scene argument block must fit the fixed-size scratch slots");

int mixed_variant(const DevScene &S) { return (S.cwm ? kVarCwm : 0) | (S.lut_mask ? kVarLut : 0); }

cudaError_t launch_generate_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                  float *state)
{
    switch (mixed_variant(S)) {
    case 1: return mixed_generate_v1(S, M, st, n0, np, state);
    case 2: return mixed_generate_v2(S, M, st, n0, np, state);
    case 3: return mixed_generate_v3(S, M, st, n0, np, state);
    default: return mixed_generate_v0(S, M, st, n0, np, state);
    }
}

cudaError_t launch_accumulate_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                    void *iq, harm_dtype dtype)
{
    switch (mixed_variant(S)) {
    case 1: return mixed_accumulate_v1(S, M, st, n0, np, iq, dtype);
    case 2: return mixed_accumulate_v2(S, M, st, n0, np, iq, dtype);
    case 3: return mixed_accumulate_v3(S, M, st, n0, np, iq, dtype);
    default: return mixed_accumulate_v0(S, M, st, n0, np, iq, dtype);
    }
}

cudaError_t launch_adjoint_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                 const void *resid, harm_dtype dtype, double *g_sigma, double *g_uv)
{
    switch (mixed_variant(S)) {
    case 1: return mixed_adjoint_v1(S, M, st, n0, np, resid, dtype, g_sigma, g_uv);
    case 2: return mixed_adjoint_v2(S, M, st, n0, np, resid, dtype, g_sigma, g_uv);
    case 3: return mixed_adjoint_v3(S, M, st, n0, np, resid, dtype, g_sigma, g_uv);
    default: return mixed_adjoint_v0(S, M, st, n0, np, resid, dtype, g_sigma, g_uv);
    }
}

cudaError_t launch_probe_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np, int *bins,
                               void *speckle, void *words, int *cells)
{
    switch (mixed_variant(S)) {
    case 1: return mixed_probe_v1(S, M, st, n0, np, bins, speckle, words, cells);
    case 2: return mixed_probe_v2(S, M, st, n0, np, bins, speckle, words, cells);
    case 3: return mixed_probe_v3(S, M, st, n0, np, bins, speckle, words, cells);
    default: return mixed_probe_v0(S, M, st, n0, np, bins, speckle, words, cells);
    }
}

int mixed_batch_pulses() { return NBG; }

// ---------------------------------------------------------------------------
// Batched persistent launch (host side)
// ---------------------------------------------------------------------------
size_t batch_args_bytes() { return sizeof(MixedArgs); }

void batch_fill_args(const harm_scene *s, void *dst, int window)
{
    MixedArgs A = make_args(s->dev, s->mixed);
    if (window == s->mixed.alt_nb) {
        A.tc = s->mixed.alt_tc;
        A.tau = s->mixed.alt_tau;
        A.nb = s->mixed.alt_nb;
        A.n_batches = s->mixed.alt_n_batches;
    }
    memcpy(dst, &A, sizeof(MixedArgs));
}

int batch_windows(const harm_scene *s, int window)
{
    return window == s->mixed.alt_nb ? s->mixed.alt_n_batches : s->mixed.n_batches;
}

int batch_tiles(const harm_scene *s, int ty)
{
    return ((s->desc.nx + TX - 1) / TX) * ((s->desc.ny + ty - 1) / ty);
}

int batch_variant(const harm_scene *s) { return mixed_variant(s->dev); }

bool batch_share3(const harm_scene *s) { return s->dev.nc == 6 && s->dev.rx_share == 0x36u; }

int batch_ctas(int device, int variant)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return ((variant & kVarCwm) ? 1 : 2) * sms;
}

cudaError_t batch_launch(const BatchLaunch &L, cudaStream_t st)
{
    switch (L.variant) {
    case 1: return mixed_batch_v1(L, st);
    case 2: return mixed_batch_v2(L, st);
    case 3: return mixed_batch_v3(L, st);
    default: return mixed_batch_v0(L, st);
    }
}

}  // namespace harm
