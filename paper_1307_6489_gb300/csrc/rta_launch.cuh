// Launch-argument blocks of the librta kernels and their host-side launchers.
#pragma once

#include "rta_device.cuh"

namespace rta {

struct ChainArgs {
    DevArray arr;
    ProcParams pp;
    const uint16_t* wave;
    int64_t n_wave;          // samples in wave
    const int64_t* wave_off;
    const int32_t* img_tel;
    const int64_t* pix_off;  // integrate-only mode, and the rows of mask_out
    int64_t n_q;             // rows of q_out / t_out / mask_out
    int64_t n_img;           // images (capacity when n_img_dev is set)
    const int64_t* n_img_dev;  // optional device-resident image count (<= n_img), read at run time
    float* q_out;            // integrate-only mode
    float* t_out;
    rta_hillas_t* out;       // full mode
    uint8_t* mask_out;       // full mode, optional: cleaning masks (general instantiations only)
    unsigned int* counter;   // zeroed before the launch
    unsigned int* status;
    int stage_wave_bytes;    // multiple of 128
    int nstage;
    int integrate_only;
    // a byte-stream bundle (rta_ingest's directory): wave is the stream, wave_off unused;
    // smeta: one prepared record per image (k_stream_meta)
    const rta_segment_t* seg;
    const int32_t* img_seg;
    int64_t n_seg;
    const struct StreamImg* smeta;
};

// One image of a byte stream as the image kernel's producer needs it: checked
// once (its segments tile the camera's pixels with 16-byte-aligned runs inside
// the stream) and read with two 16-byte loads at the image boundary; the first
// STREAM_INLINE_SEGS segments inline, the rest from the directory.
constexpr int STREAM_INLINE_SEGS = 4;
struct StreamImg {
    int ok, cam, nseg, seg0;
    long long row;               // first calibration row of the telescope
    int P, S;
    int first[STREAM_INLINE_SEGS];
    int n[STREAM_INLINE_SEGS];
    long long off[STREAM_INLINE_SEGS];
};
cudaError_t launch_stream_meta(const ChainArgs& a, StreamImg* out, int64_t max_img, int n_sm, cudaStream_t s);

struct CleanArgs {
    DevArray arr;
    ProcParams pp;
    const float* q;
    int64_t n_q;
    const int32_t* img_tel;
    const int64_t* pix_off;
    int64_t n_img;
    uint8_t* mask;
    unsigned int* status;
};

struct HillasArgs {
    DevArray arr;
    const float* q;
    const float* t;
    const uint8_t* mask;
    int64_t n_q;
    const int32_t* img_tel;
    const int64_t* pix_off;
    int64_t n_img;
    rta_hillas_t* out;
    unsigned int* status;
};

struct StereoArgs {
    DevArray arr;
    const rta_hillas_t* h;
    const int32_t* img_tel;
    int64_t n_img;
    const int32_t* evt_off;
    int64_t n_evt;             // events (capacity when n_evt_dev is set)
    const int64_t* n_img_dev;  // optional device-resident counts, read at run time
    const int64_t* n_evt_dev;
    rta_stereo_t* out;
    unsigned int* status;
    int settled;               // event offsets and counts were written before the kernel this one follows
                               // on the stream started: they are read before the dependency wait
};

int chain_variant_warps(int v);
int chain_variant_ppt(int v);
int chain_threads(int v);
int chain_stage_wave_bytes(int v, int max_S);
size_t chain_smem_bytes(int v, int nstage, int stage_wave_bytes, int max_P, int nb_keys = 0, int stream_recs = 0);
int chain_chunk_pixels(int v, int stage_wave_bytes, int S);
// which instantiation family of the fused kernel a launch uses (the occupancy of
// a family's general instantiation stands for its lean ones: same launch bounds,
// same shared memory)
enum { CHAIN_PLAIN = 0, CHAIN_NB = 1, CHAIN_STREAM = 2 };
int chain_occupancy(int v, size_t smem, int kind = CHAIN_PLAIN);
// the neighbour-peak instantiations (k_image_nb.cu), the lean ones of the image chain on
// contiguous bundles -- flat window, neighbour-peak window, digital filter -- (k_image_lean.cu)
// and the byte-stream ones (k_image_stream.cu)
cudaError_t dispatch_image_chain_nb(int v, const ChainArgs& a, int grid, size_t smem, cudaStream_t s, bool occ_only,
                                    int* occ);
cudaError_t dispatch_image_chain_lean(int v, const ChainArgs& a, int grid, size_t smem, cudaStream_t s,
                                      bool occ_only, int* occ);
cudaError_t dispatch_image_chain_stream(int v, const ChainArgs& a, int grid, size_t smem, cudaStream_t s,
                                        bool occ_only, int* occ);
int chain_variant_min_blocks(int v);
int stereo_events_per_block();
cudaError_t launch_image_chain(int v, const ChainArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_clean(const CleanArgs& a, int grid, cudaStream_t s);
cudaError_t launch_hillas(const HillasArgs& a, int grid, cudaStream_t s);
cudaError_t launch_stereo(const StereoArgs& a, int grid, cudaStream_t s);
cudaError_t launch_wait_selftest(unsigned int* status, uint64_t timeout_ns, unsigned long long* waited_ns,
                                 cudaStream_t s);
// stores a message for rta_last_error() on the calling thread
void set_last_error(const char* msg);
// sky map and geometric event rows (k_skymap.cu)
cudaError_t launch_skymap_fill(const rta_event_t* ev, int64_t n_evt, unsigned int* slab, unsigned int* slab_min,
                               cudaStream_t s);
// One window of the transient search (k_skymap.cu): counts from the ring,
// row prefix sums, disk sums, significance, alerts.
struct TransientArgs {
    const unsigned int* slabs;
    int n_slabs;
    unsigned long long use_on, use_off;
    unsigned int *on, *off, *pre_on, *pre_off;   // [256*256], [256*257] work maps
    const int* hw;                               // [2R + 1] disk half-widths
    int R;
    double alpha, s_min;
    int window;
    rta_alert_t* alerts;                         // nullable
    unsigned int* n_alerts;
    unsigned int cap;
    double* sig;                                 // nullable
    int64_t *d_on, *d_off;                       // nullable
};
cudaError_t launch_transient(const TransientArgs& t, cudaStream_t s);
cudaError_t launch_skymap_sum(const unsigned int* slabs, unsigned long long use, unsigned int* out, cudaStream_t s);
cudaError_t launch_stereo_to_events(const rta_stereo_t* st, int64_t n_evt, rta_event_t* ev, cudaStream_t s);
// DL0 byte-stream ingest (k_ingest.cu).
struct IngChunk {            // one 1 MiB piece of the stream
    long long first;         // its first packet (-1: none found)
    long long end;           // where its walk stopped (>= the piece's end, or a fault)
    long long base;          // packets in the pieces before it
    long long err_pos;
    int count;               // packets that start in it
    int err;
};
struct IngHdr {
    long long n_pk;          // packets on the chain (before a framing fault)
    long long first_bad_pk;  // earliest packet with a fault
    long long walk_err_pos;
    int walk_err;
    int error;
};
struct IngestArgs {
    DevArray arr;
    const uint8_t* stream;
    int64_t n_bytes;
    int64_t n_chunks;
    IngChunk* chunks;
    IngHdr* hdr;
    int64_t* pk_off;             // seg_cap + 1
    int* pk_err;
    unsigned long long* pk_scan;
    unsigned long long* blk_sum;
    rta_segment_t* seg;
    int64_t seg_cap;
    int32_t* img_seg;
    int32_t* img_tel;
    int64_t img_cap;
    int32_t* evt_off;
    uint64_t* evt_number;
    int64_t* evt_time;
    int64_t evt_cap;
    int64_t* counts;
    unsigned int* status;
};
int64_t ingest_chunks(int64_t n_bytes);
cudaError_t launch_ingest(const IngestArgs& a, int verify_crc, int n_sm, cudaStream_t s);

// Lookup-table reconstruction and its training sums (k_lut.cu).
struct LutArgs {
    DevArray arr;
    const rta_hillas_t* h;
    const int32_t* img_tel;
    int64_t n_img;
    const int32_t* evt_off;
    int64_t n_evt;
    const rta_stereo_t* stereo;     // reconstruction: the cores
    const float* log_e;             // training: true log10 E per event
    const float* core_xy;           // training: true impact point per event
    const uint8_t* use;             // training: events to take (nullable)
    const float* size_edges;
    int n_size;
    const float* dist_edges;
    int n_dist;
    const unsigned char* lookup;    // reconstruction: the table in lookup form (RTA_LUT_LOOKUP_BYTES a cell)
    double* acc;                    // training sums, 8 per cell
    float cut[4];                   // mscw_lo, mscw_hi, mscl_lo, mscl_hi
    rta_lut_event_t* out;
    unsigned int* status;
    int events_per_block;
};
int lut_events_per_block(int64_t n_evt, int n_sm);
cudaError_t launch_lut_reconstruct(const LutArgs& a, int grid, cudaStream_t s);
cudaError_t launch_lut_accumulate(const LutArgs& a, int grid, cudaStream_t s);
cudaError_t launch_lut_finalize(const double* acc, int64_t n_cells, int min_count, rta_lut_cell_t* cells, int grid,
                                cudaStream_t s);
cudaError_t launch_lut_prepare(const rta_lut_cell_t* cells, int64_t n_cells, void* lookup, int grid, cudaStream_t s);
// Sky-map bin of a direction coordinate: floor((v + 2.56) * 50) in FP32 with
// round-to-nearest and no contraction, -1 outside [0, RTA_SKY_N) (and for NaN).
__device__ __forceinline__ int sky_bin(float v) {
    const float u = __fmul_rn(__fadd_rn(v, 2.56f), 50.0f);
    if (!(u >= 0.f) || !(u < float(RTA_SKY_N))) return -1;
    return int(floorf(u));
}

// The event row of a geometric reconstruction: its direction, no energy or
// gamma/hadron score (NaN), no direction when the intersection is invalid.
__device__ __forceinline__ rta_event_t stereo_event_row(const rta_stereo_t& s) {
    rta_event_t r = {};
    r.log_energy = __int_as_float(0x7fc00000);
    r.gammaness = __int_as_float(0x7fc00000);
    r.dir_x = s.dir_x;
    r.dir_y = s.dir_y;
    r.n_used = s.n_valid;
    r.flags = (s.flags & RTA_SF_INVALID) ? RTA_EF_NO_DIRECTION : 0u;
    return r;
}

// context access for the surrogate (rta_api.cu)
int surrogate_ctx_tables(rta_ctx* c, const int32_t** tel_cam, const float2** tel_xy, int* n_tel, int* device);
// the context's device status word
unsigned int* surrogate_ctx_status(rta_ctx* c);
// The serving loop's passes over a batch gathered on the device (capacities and device
// counts; the counts and tables were written before the image kernel started):
// rta_server.cu calls them, rta_api.cu and rta_surrogate.cu define them.
int serve_image_chain(rta_ctx* c, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                      const int32_t* d_img_tel, const int64_t* d_n_img, int64_t max_img, int window_mode, int start,
                      int W, float t_hi, float t_lo, int core_nb, rta_hillas_t* d_out, cudaStream_t s);
int serve_stereo(rta_ctx* c, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t max_img,
                 const int32_t* d_evt_off, int64_t max_evt, const int64_t* d_n_img, const int64_t* d_n_evt,
                 rta_stereo_t* d_out, cudaStream_t s);
int serve_infer(rta_model* md, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t max_img,
                const int32_t* d_evt_off, int64_t max_evt, const int64_t* d_n_img, const int64_t* d_n_evt,
                float fallback_deg, rta_event_t* d_out, cudaStream_t s);
// Host-side check of a bundle's image table against the registered cameras: every
// offset non-negative, a multiple of 8 samples, the image inside n_wave samples; every
// telescope registered. RTA_OK or RTA_E_INVALID / RTA_E_ALIGN with the message set.
int check_bundle_images(rta_ctx* c, const int64_t* h_wave_off, const int32_t* h_img_tel, int64_t n_img,
                        int64_t n_wave);
}  // namespace rta
