// Bounds checks of the debug build (-DGAME_CHECKS).
//
// GAME_IN_BOUNDS(cond, site, idx) is true when cond holds.  In the checked build a
// failing condition also records (site, idx) in this translation unit's check word
// -- the first failure wins -- and the caller skips the access it guards; nothing
// traps, so the context stays usable and the host turns the record into
// GAME_ERR_CHECK with the site and the offending index.  Without GAME_CHECKS the
// macro is the bare condition for guards the kernel needs anyway, or `true` through
// GAME_IN_BOUNDS_DBG for checks of invariants that valid launches always satisfy.
//
// Each .cu file is its own device module (no relocatable device code), so every
// file that checks has its own word and defines a reader with
// GAME_DEFINE_CHECK_READER(name); api.cu calls the readers after each synchronising
// call.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Sites (which guard failed).
enum : int {
  kSiteExpandRow = 1,
  kSiteExpandCol = 2,
  kSitePrepareRow = 3,
  kSitePrepareSrc = 4,
  kSiteBreedParent = 5,
  kSiteBreedSlot = 6,
  kSiteSimtPartial = 7,
  kSiteOtfPartial = 8,
  kSiteTcPartial = 9,
  kSiteTcTile = 10,
  kSiteRankIndex = 11,
  kSiteScoreRow = 12,
};

#ifdef GAME_CHECKS
static __device__ unsigned long long g_game_check_word;

__device__ __forceinline__ bool game_check_record(bool ok, int site, long long idx) {
  if (!ok)
    atomicCAS(&g_game_check_word, 0ull,
              ((unsigned long long)site << 48) | ((unsigned long long)idx & 0xFFFFFFFFFFFFull));
  return ok;
}
#define GAME_IN_BOUNDS(cond, site, idx) game_check_record((cond), (site), (long long)(idx))
#define GAME_IN_BOUNDS_DBG(cond, site, idx) game_check_record((cond), (site), (long long)(idx))
// Reads and clears this file's check word: 0, or site << 48 | index.
#define GAME_DEFINE_CHECK_READER(name)                                                    \
  unsigned long long name() {                                                             \
    unsigned long long w = 0, z = 0;                                                      \
    if (cudaMemcpyFromSymbol(&w, g_game_check_word, sizeof(w)) != cudaSuccess) {          \
      cudaGetLastError();                                                                 \
      return 0;                                                                           \
    }                                                                                     \
    if (w) cudaMemcpyToSymbol(g_game_check_word, &z, sizeof(z));                          \
    return w;                                                                             \
  }
#else
#define GAME_IN_BOUNDS(cond, site, idx) (cond)
#define GAME_IN_BOUNDS_DBG(cond, site, idx) true
#define GAME_DEFINE_CHECK_READER(name) \
  unsigned long long name() { return 0; }
#endif
