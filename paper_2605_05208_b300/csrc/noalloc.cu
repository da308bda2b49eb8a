// noalloc.cu -- md_eval_leaders_noalloc: neighbourhood evaluation that allocates nothing.
//
// Some callers cannot call cudaMalloc: a host whose device memory is budgeted up front (a later
// allocation could fail or block behind another user of the GPU), a latency-critical loop that
// must not enter the allocator, or code that is only handed raw device buffers by its caller.
// For them this entry point evaluates the whole neighbourhood of one operator per solution and
// writes each solution's leader into device buffers the caller owns.  Its scratch -- the
// per-warp leader candidates and the per-solution scored-move counters -- lives in the
// file-scope device array below, which every GPU that loads the library holds until the process
// exits.
#include <mutex>

#include "mdls_internal.cuh"

// Upper bound of the scratch: n_sol * (leader records * 16 + 8) bytes must fit (1 MiB), with one
// leader record per evaluation warp: 8 * min(ceil(n_customers * wpc / 8), 1024) records, where
// wpc = min(max(n_customers / 256, 1), 8) warps share a customer on full neighbourhoods.
#define MD_NOALLOC_SCRATCH_BYTES (1u << 20)
#define MD_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[MD_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch, per device.  In host code the array's name is only a
// host-side stand-in, so the address is asked for once per device and kept here.
std::mutex g_setup_mutex;
void *g_scratch_ptr[MD_NOALLOC_MAX_DEVICES] = {nullptr};

// Operators outside [0, MD_N_OPS) skip their solution, like a negative operator: the high
// bits of ops[s] are the descent's internal flags and must not reach the evaluation.
__global__ void k_noalloc_set_ops(DevSols D, const int32_t *ops) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < D.S) D.ops[s] = (ops[s] >= 0 && ops[s] < MD_N_OPS) ? ops[s] : -1;
}

// Leader per solution (one block per solution) from the per-warp candidates in the scratch.
__global__ void k_noalloc_leaders(DevSols D, const LeadRec *lpart, int nblk, const unsigned long long *nscored,
                                  uint64_t *ids, double *fs, int64_t *n_scored) {
    const int s = blockIdx.x;
    double f;
    uint32_t id;
    int valid;
    block_leader(lpart + (size_t)s * nblk, nblk, f, id, valid);
    if (threadIdx.x == 0) {
        ids[s] = valid ? (((uint64_t)(D.ops[s] & MD_OP_MASK) << 32) | id) : 0ull;
        fs[s] = valid ? f : 0.0;
        n_scored[s] = (int64_t)nscored[s];
    }
}

}  // namespace

extern "C" md_status md_eval_leaders_noalloc(md_solutions *sols, const int32_t *ops_dev, uint64_t *ids_dev,
                                             double *dF_dev, int64_t *n_scored_dev, void *stream) {
    if (!sols || !ops_dev || !ids_dev || !dF_dev || !n_scored_dev) {
        md_set_error("md_eval_leaders_noalloc: null argument");
        return MD_ERR_ARG;
    }
    const int nblk = md_eval_partials(sols);
    const size_t lbytes = (size_t)sols->n_sol * nblk * sizeof(LeadRec);
    const size_t need = lbytes + (size_t)sols->n_sol * sizeof(unsigned long long);
    if (need > MD_NOALLOC_SCRATCH_BYTES) {
        md_set_error("md_eval_leaders_noalloc: %d solutions need %zu bytes of scratch; the static limit is %u bytes",
                     sols->n_sol, need, (unsigned)MD_NOALLOC_SCRATCH_BYTES);
        return MD_ERR_CAPACITY;
    }
    int dev = 0;
    MD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MD_NOALLOC_MAX_DEVICES) {
        md_set_error("md_eval_leaders_noalloc: device %d beyond the %d supported", dev, MD_NOALLOC_MAX_DEVICES);
        return MD_ERR_ARG;
    }
    void *base = nullptr;
    {
        // the first call on a device looks up the array's device address with that device current
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return md_cuda_check(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    LeadRec *lpart = reinterpret_cast<LeadRec *>(base);
    unsigned long long *nscored = reinterpret_cast<unsigned long long *>(static_cast<unsigned char *>(base) + lbytes);
    // the array keeps the previous call's contents: the counters must start at zero; every leader
    // candidate is overwritten by the evaluation itself
    MD_CUDA(cudaMemsetAsync(nscored, 0, sizeof(unsigned long long) * sols->n_sol, st));
    k_noalloc_set_ops<<<(sols->n_sol + 127) / 128, 128, 0, st>>>(sols->d, ops_dev);
    MD_CUDA(cudaGetLastError());
    md_moves view = {};
    view.sols = sols;
    view.d.nblk = nblk;
    view.d.lpart = lpart;
    view.d.nscored = nscored;
    md_status r = md_launch_eval(sols, &view, 0u, st);
    if (r != MD_OK) return r;
    k_noalloc_leaders<<<sols->n_sol, 256, 0, st>>>(sols->d, lpart, nblk, nscored, ids_dev, dF_dev, n_scored_dev);
    MD_CUDA(cudaGetLastError());
    return MD_OK;
}
