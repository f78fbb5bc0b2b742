// Dispatch of the FP32 spectral-energy kernel on the cube side L and the tile shape.
#include "sal_internal.cuh"

namespace sal {

cudaError_t launch_energy_fp32_l3(const EVolDesc *vols, int n, int bnd, int shape, bool persistent, cudaStream_t s);
cudaError_t launch_energy_fp32_l5(const EVolDesc *vols, int n, int bnd, int shape, bool persistent, cudaStream_t s);
cudaError_t launch_energy_fp32_l7(const EVolDesc *vols, int n, int bnd, int shape, bool persistent, cudaStream_t s);
cudaError_t launch_energy_fp32_l9(const EVolDesc *vols, int n, int bnd, int shape, bool persistent, cudaStream_t s);
cudaError_t launch_energy_fp32_l11(const EVolDesc *vols, int n, int bnd, int shape, bool persistent, cudaStream_t s);
cudaError_t launch_energy_fp32_l13(const EVolDesc *vols, int n, int bnd, int shape, bool persistent, cudaStream_t s);
cudaError_t launch_energy_fp32_l15(const EVolDesc *vols, int n, int bnd, int shape, bool persistent, cudaStream_t s);

namespace {
struct ShapeList {
    int L;
    TileShape s[kMaxShapes];
};
// Candidate tile shapes (BT x BX x BY output voxels per CTA, staging mode) per cube side;
// index 0 is the default when the autotuner has not chosen: the fastest on a 256^3 volume
// (and, for L = 7, on the 462 x 951 x 651 volume) in a measured sweep of the candidates.  The order must match the
// switch of each energy_fp32_l*.cu.
const ShapeList kShapes[] = {
    {3, {{2, 8, 32, 0}, {4, 8, 32, 0}, {2, 16, 32, 0}}},
    {5, {{2, 8, 32, 0}, {1, 8, 32, 0}, {2, 16, 32, 0}}},
    {7, {{2, 8, 32, 4}, {2, 8, 32, 0}, {2, 16, 32, 0}, {2, 8, 32, 3}, {1, 16, 32, 0}, {2, 8, 32, 2}}},
    {9, {{2, 8, 32, 4}, {2, 8, 32, 0}, {2, 16, 32, 0}, {1, 16, 32, 0}}},
    {11, {{2, 16, 32, 0}, {1, 16, 32, 0}, {1, 8, 32, 0}}},
    {13, {{2, 8, 32, 0}, {1, 16, 32, 0}, {1, 8, 32, 0}}},
    {15, {{2, 8, 32, 0}, {1, 16, 32, 0}, {1, 8, 32, 0}}},
};
const ShapeList *shapes_of(int L)
{
    for (const ShapeList &s : kShapes)
        if (s.L == L) return &s;
    return nullptr;
}
}  // namespace

int energy_num_shapes(int L)
{
    const ShapeList *s = shapes_of(L);
    if (!s) return 0;
    int n = 0;
    while (n < kMaxShapes && s->s[n].bt > 0) ++n;
    return n;
}

TileShape energy_shape(int L, int idx)
{
    const ShapeList *s = shapes_of(L);
    if (!s || idx < 0 || idx >= energy_num_shapes(L)) return TileShape{0, 0, 0, 0};
    return s->s[idx];
}

cudaError_t launch_energy_fp32_batch(const EVolDesc *vols, int n, int L, int bnd, int shape, bool persistent,
                                     cudaStream_t s)
{
    switch (L) {
        case 3: return launch_energy_fp32_l3(vols, n, bnd, shape, persistent, s);
        case 5: return launch_energy_fp32_l5(vols, n, bnd, shape, persistent, s);
        case 7: return launch_energy_fp32_l7(vols, n, bnd, shape, persistent, s);
        case 9: return launch_energy_fp32_l9(vols, n, bnd, shape, persistent, s);
        case 11: return launch_energy_fp32_l11(vols, n, bnd, shape, persistent, s);
        case 13: return launch_energy_fp32_l13(vols, n, bnd, shape, persistent, s);
        case 15: return launch_energy_fp32_l15(vols, n, bnd, shape, persistent, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_energy_tc_l3(const EVolDesc *vols, int n, int bnd, int prec, bool persistent, const TcControl &c, cudaStream_t s);
cudaError_t launch_energy_tc_l5(const EVolDesc *vols, int n, int bnd, int prec, bool persistent, const TcControl &c, cudaStream_t s);
cudaError_t launch_energy_tc_l7(const EVolDesc *vols, int n, int bnd, int prec, bool persistent, const TcControl &c, cudaStream_t s);
cudaError_t launch_energy_tc_l9(const EVolDesc *vols, int n, int bnd, int prec, bool persistent, const TcControl &c, cudaStream_t s);
cudaError_t launch_energy_tc_l11(const EVolDesc *vols, int n, int bnd, int prec, bool persistent, const TcControl &c, cudaStream_t s);
cudaError_t launch_energy_tc_l13(const EVolDesc *vols, int n, int bnd, int prec, bool persistent, const TcControl &c, cudaStream_t s);
cudaError_t launch_energy_tc_l15(const EVolDesc *vols, int n, int bnd, int prec, bool persistent, const TcControl &c, cudaStream_t s);

cudaError_t launch_energy_fp32_list_l3(const float *V, sal_dims d, int bnd, const int64_t *list, const int *count, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_list_l5(const float *V, sal_dims d, int bnd, const int64_t *list, const int *count, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_list_l7(const float *V, sal_dims d, int bnd, const int64_t *list, const int *count, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_list_l9(const float *V, sal_dims d, int bnd, const int64_t *list, const int *count, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_list_l11(const float *V, sal_dims d, int bnd, const int64_t *list, const int *count, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_list_l13(const float *V, sal_dims d, int bnd, const int64_t *list, const int *count, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_list_l15(const float *V, sal_dims d, int bnd, const int64_t *list, const int *count, float *E, cudaStream_t s);

// Shape-0 tiles of a device-side list (the surrogate's fallback).
cudaError_t launch_energy_fp32_list(const float *V, sal_dims d, int L, int bnd, const int64_t *list, const int *count,
                                    float *E, cudaStream_t s)
{
    switch (L) {
        case 3: return launch_energy_fp32_list_l3(V, d, bnd, list, count, E, s);
        case 5: return launch_energy_fp32_list_l5(V, d, bnd, list, count, E, s);
        case 7: return launch_energy_fp32_list_l7(V, d, bnd, list, count, E, s);
        case 9: return launch_energy_fp32_list_l9(V, d, bnd, list, count, E, s);
        case 11: return launch_energy_fp32_list_l11(V, d, bnd, list, count, E, s);
        case 13: return launch_energy_fp32_list_l13(V, d, bnd, list, count, E, s);
        case 15: return launch_energy_fp32_list_l15(V, d, bnd, list, count, E, s);
        default: return cudaErrorInvalidValue;
    }
}

bool energy_tc_supported(int L, int prec)
{
    if (prec == SAL_PREC_BF16) return L >= 3 && L <= 15 && (L & 1);
    if (prec == SAL_PREC_TF32) return L >= 3 && L <= 11 && (L & 1);
    return false;
}

cudaError_t launch_energy_tc(const EVolDesc *vols, int n, int L, int bnd, int prec, bool persistent,
                             const TcControl &c, cudaStream_t s)
{
    if (!energy_tc_supported(L, prec)) return cudaErrorInvalidValue;
    switch (L) {
        case 3: return launch_energy_tc_l3(vols, n, bnd, prec, persistent, c, s);
        case 5: return launch_energy_tc_l5(vols, n, bnd, prec, persistent, c, s);
        case 7: return launch_energy_tc_l7(vols, n, bnd, prec, persistent, c, s);
        case 9: return launch_energy_tc_l9(vols, n, bnd, prec, persistent, c, s);
        case 11: return launch_energy_tc_l11(vols, n, bnd, prec, persistent, c, s);
        case 13: return launch_energy_tc_l13(vols, n, bnd, prec, persistent, c, s);
        case 15: return launch_energy_tc_l15(vols, n, bnd, prec, persistent, c, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_energy_fp32(const float *V, sal_dims d, int L, int bnd, float *E, cudaStream_t s)
{
    EVolDesc v{V, E, d.T, d.X, d.Y};
    return launch_energy_fp32_batch(&v, 1, L, bnd, 0, false, s);
}

}  // namespace sal
