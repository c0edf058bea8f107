// Registry of compiled instantiations of the fused f/grad kernel.
#pragma once
#include <cuda.h>

namespace rpca {

struct FgArgs;
typedef void (*FgKernelFn)(const CUtensorMap, const CUtensorMap, FgArgs);

struct FgVariant {
  const void* fn;  // __global__ function pointer (nullptr: not compiled)
  int R;           // rows per lane
  int J;           // columns per reduction group
  // Grouped form of the same instantiation (fg_group_kernel: many problems' tiles in one
  // launch), nullptr when not compiled: fg mode, unmasked, float32 X.
  const void* group = nullptr;
};

// Forming rank K (0..16), product width B, fg mode (B == K, operands = forming factors) or
// apply mode with side 0 (both products), 1 (D Bv only) or 2 (D^T Bu only), masked or not
// (apply mode: B = 8, or B = 16 with K = 0 on sides 1 and 2).
// Returns nullptr when that combination is not compiled.
// xt: storage type of X (0 float32, 1 bfloat16, 2 FP8 E4M3); narrow storage is compiled for
// fg mode with K <= 8 only.
const FgVariant* fg_variant(int K, int B, bool same, bool masked, int side = 0, int xt = 0);

void fg_register_same_small(FgVariant (*tab)[2]);   // K = 1..8
void fg_register_same_large(FgVariant (*tab)[2]);   // K = 9..16
void fg_register_same_bf16(FgVariant (*tab)[2]);    // K = 1..8, X stored as bfloat16
void fg_register_same_e4m3(FgVariant (*tab)[2]);    // K = 1..8, X stored as FP8 E4M3
void fg_register_apply(FgVariant (*tab)[3][2]);     // K = 0, 8, 16; B = 8; three sides
void fg_register_apply16(FgVariant (*tab)[2]);      // K = 0, B = 16; sides 1 and 2
void fg_register_mma(FgVariant* tab);               // tensor-core form, K = 1..8, fg mode, float32 X

// Tensor-core form of the fused kernel (fg_mma.cu) for forming rank K, or nullptr.
const FgVariant* fg_mma_variant(int K, bool masked);

void fg_register_tc(FgVariant* tab);  // tcgen05 form, K = 1..6, fg mode, float32 X, unmasked
// tcgen05 form (fg_tc.cu) for forming rank K, or nullptr; its shared memory for a plan.
const FgVariant* fg_tc_variant(int K, bool masked);
size_t fg_tc_smem_bytes(int BN, int K, int nstage, int J);

}  // namespace rpca
