// Internal declarations of libefe (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/efe.h"

#define EFE_MAXP 8
#define EFE_MAXNQ 12

// Device-side mesh constants passed by value to kernels.
struct MeshDev {
    int nx, ny, nz;          // cells per axis
    int Gx, Gy, Gz;          // nodes per axis
    int p, np1, ne;          // degree, p+1, (p+1)^3
    int nq, nq3;             // Gauss points per axis, nq^3
    double h;
};

// Per-(atom, cell) pair used by the projection kernels.
struct PairInfo {
    int atom;
    int cell;
};

// flags in the high bits of the node-major atom index of a coupling entry
constexpr int kNmHasE = 1 << 30, kNmHasP = 1 << 29, kNmAtomMask = (1 << 29) - 1;

struct efe_ctx {
    std::string err;
    cudaStream_t stream = nullptr;
    int device = 0;                           // CUDA device current at efe_setup (the stream's device)
    cusolverDnHandle_t solver = nullptr;
    MeshDev m{};
    int natoms = 0, n_enr = 0, n_proj = 0;
    long long n_nodes = 0, n_rows = 0, n_fe_dof = 0, n_quad = 0;
    bool enrich = false, nonlocal = false;
    double alpha = 1.2, r0 = 1.0, t = 0.33;
    double rc = 1.0, rtrunc = 6.0, rloc = 0.8;
    std::vector<double> xyz, zval, hproj;     // host copies
    bool have_potential = false;

    // --- host tables -------------------------------------------------
    std::vector<double> xg, wg, xq, wq;       // GLL and Gauss rules on [-1, 1]
    std::vector<double> B1, D1;               // nq x (p+1)

    // --- device tables -----------------------------------------------
    double *d_B1 = nullptr, *d_D1 = nullptr, *d_wq = nullptr;   // 1D tables
    double *d_Khat = nullptr;                 // ne x ne, 1/2 K_e for this h
    double *d_mcc = nullptr, *d_minv = nullptr;  // n_nodes (0 on boundary for minv)
    double *d_He = nullptr;                   // n_cells x ne x ne, FP64
    float *d_He32 = nullptr;                  // n_cells x ne x ne, FP32 copy
    void *d_He16 = nullptr;                   // bf16 tiles for the tensor-core path
    size_t he16_bytes = 0;
    bool he16_valid = false;                  // tiles match the current potential
    double *d_atoms = nullptr;                // natoms x 3
    double *d_hproj = nullptr;                // n_proj (per projector strength)

    // supports (per atom): positions into concatenated arrays
    std::vector<long long> sup_off;           // natoms + 1
    long long *d_sup_off = nullptr;           // device copy
    long long sup_total = 0;
    int *d_sup_node = nullptr;                // sup_total
    double *d_C = nullptr;                    // sup_total x 4  (C_I[pos][f])
    double *d_B = nullptr;                    // sup_total x 4
    double *d_Kca = nullptr;                  // sup_total x 4 (1/2 grad N . grad a)
    double *d_Hca = nullptr;                  // sup_total x 4 (Kca + Vca)
    double *d_Pc = nullptr;                   // sup_total x 4 (<beta_f, N_j>)
    // the FE-enrichment block of H^E itself, E = H^ac - C H^cc (sup_total x 4, per
    // potential): the mixed filter applies H^E through E instead of T^T H_raw T,
    // whose two large terms cancel when the enrichment is nearly representable
    // by the FE space
    double *d_E = nullptr;
    float *d_E32 = nullptr, *d_Pc32 = nullptr;   // FP32 copies for the mixed filter
    // the same in node-major (CSR) order, with the atom of each entry, for the node kernels
    int *d_nm_atom = nullptr;                 // atom | kNmHasE | kNmHasP
    float *d_nm_E32 = nullptr, *d_nm_P32 = nullptr;
    // launch order of the support reductions' (atom, chunk) blocks, by first node
    int2 *d_chunk_order = nullptr;
    int chunk_order_nch = 0;
    // node -> (atom, pos) CSR over all nodes
    long long *d_node_ptr = nullptr;          // n_nodes + 1
    int *d_node_ent = nullptr;                // entries: global support index (sup_off[I] + pos)
    int *d_ent_atom = nullptr;                // atom of each support entry
    // pairs
    std::vector<PairInfo> pairs;              // sorted by cell colour
    std::vector<int> pair_colour_off;         // 9 offsets
    PairInfo *d_pairs = nullptr;
    int *d_pair_pos = nullptr;                // npairs x ne : support position or -1
    // cell -> atoms
    int *d_cell_atom_ptr = nullptr, *d_cell_atoms = nullptr;
    // dense enriched blocks (n_enr x n_enr), projector blocks
    double *d_Aee = nullptr, *d_Kaa = nullptr, *d_Haa = nullptr, *d_Mee = nullptr;
    double *d_Pa = nullptr;                   // n_proj x n_enr
    double *d_PE = nullptr;                   // n_proj x n_enr: <beta_p, N^E_k> = Pa - Pc C^T
    double *d_HEee = nullptr;                 // n_enr x n_enr: H^E_ee (local part), per potential
    double *d_Mblk_inv = nullptr;             // natoms x 16
    double *d_Mblk = nullptr;                 // natoms x 16

    // --- workspaces (grown on demand) -----------------------------------
    size_t ws_bytes = 0;
    void *d_ws = nullptr;
    size_t part_bytes = 0;
    double *d_part = nullptr;                 // partial sums
    double *h_pinned = nullptr;
    size_t pinned_bytes = 0;
    int *d_info = nullptr;
    int *d_err = nullptr;                     // device error flag of bounded waits
    void *d_solver_ws = nullptr;
    size_t solver_ws_bytes = 0;

    efe_stats stats{};
    long long launches = 0;
    void *scf = nullptr;                      // SCF buffers (efe_scf.cu), freed by efe_destroy
    // cell-product timing: events recorded around each colour sweep, summed
    // after the next synchronisation of the stream
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> cell_events;
    size_t cell_events_used = 0;
    // the same for the node-recurrence kernels of the bf16 filter
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> rec_events;
    size_t rec_events_used = 0;
    long long n_support_nodes = 0;
    // device copies for the host-buffer filter (grown on demand, kept)
    void *d_hostio = nullptr;
    size_t hostio_bytes = 0;
    long long cell_launches = 0;
    bool cells_bf16 = true;                   // mixed filter: per-cell products stored in bf16 (else FP32)
    int poisson_mixed = -1;                   // Poisson CG: 1 FP32 refinement stage, 0 FP64 only, -1 by mesh size
    // coupling as extra k-steps of the tensor-core cell products (efe_tc.cu)
    bool cx_built = false;
    int *d_cx_off = nullptr;                  // n_cells + 1: first extra k-step of each cell
    int *d_cx_atoms = nullptr;                // two atom slots per extra k-step (natoms: zero block)
    void *d_Ax = nullptr;                     // extra A stages, bf16 [k-step][MT][2048]
    long long cx_steps = 0;
    int cx_max_slots = 0;                     // largest atom-slot count of a cell
    // E Y_c from the padding rows of the cell products (rows ne .. MT*128 of the
    // last M-tile hold, per atom slot, the E coefficients of the owned nodes)
    bool epad = false;
    int *d_atom_pair_off = nullptr;           // natoms + 1
    int *d_atom_pairs = nullptr;              // per atom: its (cell, atom) pairs (indices into d_cell_atoms)
    int ca_pairs = 0;                         // number of (cell, atom) support pairs
    // the support entries with a nonzero projector row, per atom (sorted by node)
    std::vector<long long> psup_off;          // natoms + 1
    long long *d_psup_off = nullptr;
    int *d_psup_node = nullptr;
    float *d_psup_coef = nullptr;             // 4 per entry
    int2 *d_pchunk_order = nullptr;
    int pchunk_nch = 0;
    // per atom, the atoms whose blocks of H^E_ee or P^E are not all zero (per potential)
    int *d_enbr_ptr = nullptr, *d_enbr = nullptr;
};

// error helpers
#define EFE_CUDA(ctx, call)                                                          \
    do {                                                                             \
        cudaError_t _e = (call);                                                     \
        if (_e != cudaSuccess) {                                                     \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(_e);         \
            return EFE_ERR_CUDA;                                                     \
        }                                                                            \
    } while (0)

#define EFE_TRY(call)                                                                \
    do {                                                                             \
        efe_status _s = (call);                                                      \
        if (_s != EFE_OK) return _s;                                                 \
    } while (0)

efe_status efe_check_launch(efe_ctx *ctx, const char *what);
efe_status efe_alloc(efe_ctx *ctx, void **p, size_t bytes);
efe_status efe_workspace(efe_ctx *ctx, size_t bytes);
efe_status efe_partials(efe_ctx *ctx, size_t doubles);
efe_status efe_pinned(efe_ctx *ctx, size_t bytes);

// kernels/launchers shared between translation units
efe_status efe_build_tables(efe_ctx *ctx);
efe_status efe_static_integrals(efe_ctx *ctx);
efe_status efe_potential_assembly(efe_ctx *ctx, const double *veff_q);
efe_status efe_hx(efe_ctx *ctx, const double *X, double *Y, int N, efe_precision prec,
                  double *wsXp);
efe_status efe_hx_f32(efe_ctx *ctx, const float *X, float *Y, int N, efe_precision prec);
efe_status efe_mx(efe_ctx *ctx, const double *X, double *Y, int N);
efe_status efe_minvx(efe_ctx *ctx, const double *X, double *Y, int N);
efe_status efe_tc_prepare(efe_ctx *ctx);
void efe_scf_free(efe_ctx *ctx);
efe_status efe_cells_shared(efe_ctx *ctx, const double *K, const double *X, double *Y, int N);
efe_status efe_xprime_fp64(efe_ctx *ctx, const double *X, double *Xp, int N);
void efe_sym_eig(int n, const std::vector<double> &A, std::vector<double> &w, std::vector<double> &V);
efe_status efe_tc_cells(efe_ctx *ctx, const void *Xp_bf16, int ldb, int N, void *Ycells, int ldy, int *d_err,
                        int out_bf16 = 0, const void *YW = nullptr, int nCB = 0, float *Epart = nullptr);
int efe_tc_columns(const efe_ctx *ctx, int N, int ldb);
