// Fitted-model files: the state Algorithm 2's online phase reuses (training
// features X, the neighbour table, the precomputed coefficients C, k and the
// kernel hyperparameters), so that a model outlives the process that fitted
// it.  The paper has no file format; this one is the library's own.
//
// Layout (little-endian, as both supported hosts are):
//   128-byte header (FileHeader below), then X (n x d, FP64 or FP32), the
//   neighbour table (n x nbr_ld int32), C (n x k x r, 8 bytes per
//   coefficient: FP64, or the mixed form's FP32 pairs), each row-major.
//   The checksum is FNV-1a (64-bit offset basis and prime) applied to the
//   data as 8-byte little-endian words, then to any bytes left over, over the
//   header (with its checksum field zero) followed by the three arrays.
// Arrays move between the device and the file through a pinned staging
// buffer of at most 64 MB, so a model of many GB needs no host copy.
#include <stdio.h>
#include <string.h>
#include <algorithm>
#include "model.cuh"

namespace fmgp {
namespace {

constexpr char kMagic[8] = {'F', 'M', 'G', 'P', 'M', 'O', 'D', 'L'};
constexpr uint32_t kVersion = 1;
constexpr size_t kStage = (size_t)64 << 20;

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int32_t dtype, precision;
  int64_t n;
  int32_t d, r, k, nbr_ld;
  int32_t kernel_kind, pad0;
  double nu, length_scale, variance, nugget;
  uint64_t x_bytes, nbr_bytes, c_bytes;
  uint64_t checksum;
  uint8_t reserved[8];
};
static_assert(sizeof(FileHeader) == 128, "the file header is 128 bytes");

struct Fnv {
  uint64_t h = 0xcbf29ce484222325ull;
  uint8_t tail[8];
  int ntail = 0;
  void word(uint64_t w) {
    h ^= w;
    h *= 0x100000001b3ull;
  }
  // Bytes are taken in order across calls: whole 8-byte words as they
  // complete, the last partial word byte by byte in finish().
  void add(const void* p, size_t len) {
    const uint8_t* b = (const uint8_t*)p;
    while (len && ntail) {
      tail[ntail++] = *b++;
      --len;
      if (ntail == 8) {
        uint64_t w;
        memcpy(&w, tail, 8);
        word(w);
        ntail = 0;
      }
    }
    for (; len >= 8; len -= 8, b += 8) {
      uint64_t w;
      memcpy(&w, b, 8);
      word(w);
    }
    while (len--) tail[ntail++] = *b++;
  }
  uint64_t finish() {
    for (int i = 0; i < ntail; ++i) word(tail[i]);
    ntail = 0;
    return h;
  }
};

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

struct Pinned {
  void* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

// Device array -> file (and checksum), through the staging buffer.
int write_array(FILE* f, const void* dev, uint64_t bytes, void* stage, Fnv& h, cudaStream_t s) {
  for (uint64_t off = 0; off < bytes; off += kStage) {
    const size_t len = (size_t)std::min<uint64_t>(kStage, bytes - off);
    FMGP_CUDA_TRY(cudaMemcpyAsync(stage, (const char*)dev + off, len, cudaMemcpyDeviceToHost, s));
    FMGP_CUDA_TRY(cudaStreamSynchronize(s));
    h.add(stage, len);
    if (fwrite(stage, 1, len, f) != len) {
      set_error("model file: write failed");
      return FMGP_EIO;
    }
  }
  return FMGP_OK;
}

// File -> device array (and checksum), through the staging buffer.
int read_array(FILE* f, void* dev, uint64_t bytes, void* stage, Fnv& h, cudaStream_t s) {
  for (uint64_t off = 0; off < bytes; off += kStage) {
    const size_t len = (size_t)std::min<uint64_t>(kStage, bytes - off);
    if (fread(stage, 1, len, f) != len) {
      set_error("model file: truncated (expected %llu more bytes)",
                (unsigned long long)(bytes - off));
      return FMGP_EIO;
    }
    h.add(stage, len);
    FMGP_CUDA_TRY(cudaMemcpyAsync((char*)dev + off, stage, len, cudaMemcpyHostToDevice, s));
    FMGP_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return FMGP_OK;
}

uint64_t x_bytes_of(int dtype, int64_t n, int d) {
  return (uint64_t)n * d * (dtype == FMGP_F64 ? 8 : 4);
}

}  // namespace
}  // namespace fmgp

using namespace fmgp;

extern "C" int fmgp_model_get_info(const fmgp_model* model, fmgp_model_info* out) {
  clear_error();
  const Model* m = reinterpret_cast<const Model*>(model);
  if (!m || !out) {
    set_error("model and out must be non-NULL");
    return FMGP_EINVAL;
  }
  out->n = m->n;
  out->d = m->d;
  out->r = m->r;
  out->k = m->k;
  out->nbr_ld = m->ld;
  out->dtype = m->dtype;
  out->precision = m->prec;
  out->kernel = m->kern;
  return FMGP_OK;
}

extern "C" int fmgp_model_save(const fmgp_model* model, const char* path, void* stream) {
  clear_error();
  const Model* m = reinterpret_cast<const Model*>(model);
  if (!m || !path) {
    set_error("model and path must be non-NULL");
    return FMGP_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  FileHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kMagic, 8);
  hd.version = kVersion;
  hd.header_bytes = sizeof(FileHeader);
  hd.dtype = m->dtype;
  hd.precision = m->prec;
  hd.n = m->n;
  hd.d = m->d;
  hd.r = m->r;
  hd.k = m->k;
  hd.nbr_ld = m->ld;
  hd.kernel_kind = m->kern.kind;
  hd.nu = m->kern.nu;
  hd.length_scale = m->kern.length_scale;
  hd.variance = m->kern.variance;
  hd.nugget = m->kern.nugget;
  hd.x_bytes = x_bytes_of(m->dtype, m->n, m->d);
  hd.nbr_bytes = m->k > 1 ? (uint64_t)m->n * m->ld * 4 : 0;
  hd.c_bytes = (uint64_t)m->n * m->k * m->r * 8;
  File f;
  f.f = fopen(path, "wb");
  if (!f.f) {
    set_error("model file: cannot open '%s' for writing", path);
    return FMGP_EIO;
  }
  Pinned st;
  FMGP_CUDA_TRY(cudaMallocHost(&st.p, kStage));
  // the checksum covers the header with its own field zero: write a
  // placeholder header, the arrays, then the final header over it
  if (fwrite(&hd, 1, sizeof(hd), f.f) != sizeof(hd)) {
    set_error("model file: write failed");
    return FMGP_EIO;
  }
  Fnv h;
  h.add(&hd, sizeof(hd));
  int rc = write_array(f.f, m->X, hd.x_bytes, st.p, h, s);
  if (!rc && hd.nbr_bytes) rc = write_array(f.f, m->nbr, hd.nbr_bytes, st.p, h, s);
  if (!rc) rc = write_array(f.f, m->C, hd.c_bytes, st.p, h, s);
  if (rc) return rc;
  hd.checksum = h.finish();
  if (fseek(f.f, 0, SEEK_SET) != 0 || fwrite(&hd, 1, sizeof(hd), f.f) != sizeof(hd) ||
      fflush(f.f) != 0) {
    set_error("model file: write failed");
    return FMGP_EIO;
  }
  return FMGP_OK;
}

extern "C" int fmgp_model_load(const char* path, fmgp_model** out, void* stream) {
  clear_error();
  if (!path || !out) {
    set_error("path and out must be non-NULL");
    return FMGP_EINVAL;
  }
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  File f;
  f.f = fopen(path, "rb");
  if (!f.f) {
    set_error("model file: cannot open '%s'", path);
    return FMGP_EIO;
  }
  FileHeader hd;
  if (fread(&hd, 1, sizeof(hd), f.f) != sizeof(hd) || memcmp(hd.magic, kMagic, 8) != 0) {
    set_error("model file: '%s' is not a model file", path);
    return FMGP_EIO;
  }
  if (hd.version != kVersion || hd.header_bytes != sizeof(FileHeader)) {
    set_error("model file: version %u unsupported (this library reads version %u)", hd.version,
              kVersion);
    return FMGP_EIO;
  }
  if ((hd.dtype != FMGP_F32 && hd.dtype != FMGP_F64) || hd.n < 1 || hd.n >= INT32_MAX ||
      hd.d < 1 || hd.r < 1 || hd.k < 1 || hd.k > kMaxK || hd.k > hd.n || hd.nbr_ld < hd.k - 1 ||
      hd.x_bytes != x_bytes_of(hd.dtype, hd.n, hd.d) ||
      hd.nbr_bytes != (hd.k > 1 ? (uint64_t)hd.n * hd.nbr_ld * 4 : 0) ||
      hd.c_bytes != (uint64_t)hd.n * hd.k * hd.r * 8) {
    set_error("model file: header sizes are inconsistent");
    return FMGP_EIO;
  }
  const uint64_t want = hd.checksum;
  hd.checksum = 0;
  Fnv h;
  h.add(&hd, sizeof(hd));
  void* bufs[3] = {nullptr, nullptr, nullptr};
  auto release = [&]() {
    for (void* b : bufs)
      if (b) cudaFree(b);
  };
  const uint64_t sizes[3] = {hd.x_bytes, hd.nbr_bytes, hd.c_bytes};
  for (int i = 0; i < 3; ++i) {
    if (!sizes[i]) continue;
    if (cudaMalloc(&bufs[i], sizes[i]) != cudaSuccess) {
      cudaGetLastError();
      release();
      set_error("model file: cannot allocate %llu device bytes", (unsigned long long)sizes[i]);
      return FMGP_ENOMEM;
    }
  }
  Pinned st;
  cudaError_t e = cudaMallocHost(&st.p, kStage);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "cudaMallocHost");
  }
  int rc = FMGP_OK;
  for (int i = 0; i < 3 && !rc; ++i)
    if (sizes[i]) rc = read_array(f.f, bufs[i], sizes[i], st.p, h, s);
  if (!rc && h.finish() != want) {
    set_error("model file: checksum mismatch (the file is damaged)");
    rc = FMGP_EIO;
  }
  if (rc) {
    release();
    return rc;
  }
  fmgp_kernel kern;
  kern.kind = hd.kernel_kind;
  kern.nu = hd.nu;
  kern.length_scale = hd.length_scale;
  kern.variance = hd.variance;
  kern.nugget = hd.nugget;
  void* owned[3];
  int nowned = 0;
  for (void* b : bufs)
    if (b) owned[nowned++] = b;
  return model_create(bufs[0], (fmgp_dtype)hd.dtype, hd.n, hd.d, (const int32_t*)bufs[1],
                      hd.nbr_ld, bufs[2], hd.k, hd.r, &kern, (fmgp_precision)hd.precision, out, s,
                      owned, nowned);
}
