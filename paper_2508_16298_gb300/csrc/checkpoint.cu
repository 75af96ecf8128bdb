// Checkpoint / resume of a Markov chain: a flat little-endian binary file with
// the model and lattice, the chain's position (theta, the Philox seed and the
// next trajectory counter), its step size and acceptance statistics, and
// optionally the learned net's FP32 master weights.  Host-only: the caller
// copies theta between the device and host memory.  Because every random
// number of a trajectory is a function of (seed, counter), a chain resumed from
// a checkpoint continues bit for bit as if it had never stopped.
//
// Layout: 8-byte magic "HQMCCKP1", then hqmc_checkpoint (fixed fields), then
// 2 * Ntau * L * L doubles of theta, then n_weights floats, then the 64-bit
// FNV-1a hash of everything after the magic.
#include <cstdio>
#include <cstring>
#include <vector>

#include "hqmc.h"

namespace {

constexpr char kMagic[8] = {'H', 'Q', 'M', 'C', 'C', 'K', 'P', '1'};

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
};

bool valid_header(const hqmc_checkpoint* c) {
  const long long n = (long long)c->L * c->L * c->Ntau;
  return c->L >= 4 && (c->L & 1) == 0 && c->L <= 68 && c->Ntau >= 2 && n <= (1LL << 31) - 1 && c->n_weights >= 0 &&
         c->n_weights <= (1 << 24);
}

}  // namespace

extern "C" int hqmc_checkpoint_write(const char* path, const hqmc_checkpoint* c, const double* theta_host,
                                     const float* weights_host) {
  if (!path || !c || !theta_host || !valid_header(c) || (c->n_weights > 0 && !weights_host)) return HQMC_EINVAL;
  const size_t nth = 2 * (size_t)c->L * c->L * c->Ntau;
  FILE* f = std::fopen(path, "wb");
  if (!f) return HQMC_EIO;
  Fnv h;
  h.add(c, sizeof(*c));
  h.add(theta_host, nth * sizeof(double));
  if (c->n_weights) h.add(weights_host, (size_t)c->n_weights * sizeof(float));
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(c, sizeof(*c), 1, f) == 1 &&
            std::fwrite(theta_host, sizeof(double), nth, f) == nth &&
            (c->n_weights == 0 || std::fwrite(weights_host, sizeof(float), c->n_weights, f) == (size_t)c->n_weights) &&
            std::fwrite(&h.h, sizeof(h.h), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? HQMC_OK : HQMC_EIO;
}

extern "C" int hqmc_checkpoint_read(const char* path, hqmc_checkpoint* c, double* theta_host, float* weights_host) {
  if (!path || !c) return HQMC_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return HQMC_EIO;
  char magic[8];
  hqmc_checkpoint hdr;
  int rc = HQMC_OK;
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMagic, 8) != 0 || std::fread(&hdr, sizeof(hdr), 1, f) != 1 ||
      !valid_header(&hdr)) {
    rc = HQMC_EIO;
  } else if (theta_host) {  // full read: payload and hash
    const size_t nth = 2 * (size_t)hdr.L * hdr.L * hdr.Ntau;
    std::vector<float> w(hdr.n_weights);
    uint64_t stored = 0;
    if (std::fread(theta_host, sizeof(double), nth, f) != nth ||
        (hdr.n_weights && std::fread(w.data(), sizeof(float), w.size(), f) != w.size()) ||
        std::fread(&stored, sizeof(stored), 1, f) != 1) {
      rc = HQMC_EIO;
    } else {
      Fnv h;
      h.add(&hdr, sizeof(hdr));
      h.add(theta_host, nth * sizeof(double));
      if (hdr.n_weights) h.add(w.data(), w.size() * sizeof(float));
      if (h.h != stored) rc = HQMC_EIO;
      else if (weights_host && hdr.n_weights) std::memcpy(weights_host, w.data(), w.size() * sizeof(float));
    }
  }
  std::fclose(f);
  if (rc == HQMC_OK) *c = hdr;
  return rc;
}
