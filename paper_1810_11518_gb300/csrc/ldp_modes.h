// Kernel modes and device status bits shared by the host code and the
// device code.
#pragma once

namespace ldp {

// kLDP: the k largest |m_i| (ties to the lower index), Eq. 2-3.  kLBP: Sec.
// 2.1.  The other LDP modes are the remaining readings of Eq. 2-3: kLDPRaw
// ranks the signed m_i; kLDPThresh / kLDPRawThresh apply s(x >= 0) literally
// against the k-th ranked response, so every response tied with it is set
// (k or more bits).
enum Mode { kLDP = 0, kLBP = 1, kLDPRaw = 2, kLDPThresh = 3, kLDPRawThresh = 4 };
__host__ __device__ constexpr bool is_ldp(int mode) { return mode != kLBP; }
// codes of exactly k bits (compact bins exist)
__host__ __device__ constexpr bool exact_k(int mode) { return mode == kLDP || mode == kLDPRaw; }

// Bits of the device status word (read and cleared by ldp_device_status).
constexpr int kStatusBadDesc = 1;      // a batch or window descriptor was rejected
constexpr int kStatusTooManyTiles = 2;  // a batch needed more tiles than its work list holds
constexpr int kStatusWaitTimeout = 4;  // a bounded wait for staged input gave up
constexpr int kStatusBadCrop = 8;      // a crop descriptor was rejected
constexpr int kStatusBounds = 16;      // checked builds: an index outside its buffer was skipped

}  // namespace ldp
