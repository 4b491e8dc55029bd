// Strided-pass dispatch: picks the tile width (the per-length default, or the
// width the autotuner chose in SParams::tile) and the kernel instance.
#include <mutex>

#include "spe_internal.cuh"
#include "fft_tile.cuh"
#include "tma.cuh"

namespace spe {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    });
    return fn;
}

cudaError_t launch_spass_t8(int n, const SParams &p, cudaStream_t st, int *blocks_out);
cudaError_t launch_spass_t16(int n, const SParams &p, cudaStream_t st, int *blocks_out);
cudaError_t launch_spass_t32(int n, const SParams &p, cudaStream_t st, int *blocks_out);
cudaError_t setup_spass_attributes_t8();
cudaError_t setup_spass_attributes_t16();
cudaError_t setup_spass_attributes_t32();
cudaError_t launch_spass_tc(int n, const SParams &p, cudaStream_t st, int *blocks_out);
cudaError_t setup_tc_attributes();

int spass_default_tile(int n) { return n >= 256 ? 16 : 32; }

bool has_alt_plan_n(int n)
{
    switch (n) {
#define X(n) \
    case n: return has_alt_plan<n>();
        SPE_FOR_EACH_N(X)
#undef X
    default: return false;
    }
}

int plan_count_n(int n)
{
    switch (n) {
#define X(n) \
    case n: return has_plan2<n>() ? 3 : (has_alt_plan<n>() ? 2 : 1);
        SPE_FOR_EACH_N(X)
#undef X
    default: return 1;
    }
}

bool spass_tile_ok(int n, int tile)
{
    return tile == 8 || tile == 16 || (tile == 32 && (size_t)n * 32 * 8 <= 227 * 1024);
}

cudaError_t launch_spass(int n, const SParams &p, cudaStream_t st, int *blocks_out)
{
    if (p.tc && (n == 256 || n == 512)) return launch_spass_tc(n, p, st, blocks_out);
    int tw = p.tile ? p.tile : spass_default_tile(n);
    if (!spass_tile_ok(n, tw)) tw = 16;
    if (tw == 8) return launch_spass_t8(n, p, st, blocks_out);
    return tw == 16 ? launch_spass_t16(n, p, st, blocks_out) : launch_spass_t32(n, p, st, blocks_out);
}

cudaError_t setup_spass_attributes()
{
    cudaError_t e = setup_spass_attributes_t8();
    if (e == cudaSuccess) e = setup_spass_attributes_t16();
    if (e == cudaSuccess) e = setup_spass_attributes_t32();
    if (e == cudaSuccess) e = setup_tc_attributes();
    return e;
}

}  // namespace spe
