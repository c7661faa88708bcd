// Generated by gen_fnodes.py: the UTD transition function F(X) (re, im) at X_i = 6 + i / 2,
// i = 0..68, from its continued fraction in 50-digit arithmetic.
#pragma once

namespace drt {

constexpr double FNODE_X0 = 6.0, FNODE_H = 0.5;
constexpr int FNODE_N = 69;
static __device__ const double kFnode[2 * FNODE_N] = {
    0x1.f70a59f654e58p-1, 0x1.3ab28d5b92301p-4,   // X = 6.0
    0x1.f8350a58b2d75p-1, 0x1.257004486c638p-4,   // X = 6.5
    0x1.f92a0001b778fp-1, 0x1.12c3f2b7a81fap-4,   // X = 7.0
    0x1.f9f53bbf76d1bp-1, 0x1.023f9fddf2536p-4,   // X = 7.5
    0x1.fa9f986ac1b10p-1, 0x1.e716530b13079p-5,   // X = 8.0
    0x1.fb2fbaad43b3bp-1, 0x1.ccc00b8935590p-5,   // X = 8.5
    0x1.fbaab1bb18833p-1, 0x1.b50a030301848p-5,   // X = 9.0
    0x1.fc14656658504p-1, 0x1.9f9694eb2f833p-5,   // X = 9.5
    0x1.fc6fe2f832224p-1, 0x1.8c186f84ccc17p-5,   // X = 10.0
    0x1.fcbf93c64262fp-1, 0x1.7a4f384354b12p-5,   // X = 10.5
    0x1.fd05649394676p-1, 0x1.6a04f96b7ec7ap-5,   // X = 11.0
    0x1.fd42e261886fap-1, 0x1.5b0c24a283131p-5,   // X = 11.5
    0x1.fd794fcc8153cp-1, 0x1.4d3e04f03abe8p-5,   // X = 12.0
    0x1.fda9b51297d4dp-1, 0x1.40798507c5779p-5,   // X = 12.5
    0x1.fdd4ec3b8d937p-1, 0x1.34a235eafb3edp-5,   // X = 13.0
    0x1.fdfbaa696451ep-1, 0x1.299f872678bbfp-5,   // X = 13.5
    0x1.fe1e870cf2269p-1, 0x1.1f5c259b4569ap-5,   // X = 14.0
    0x1.fe3e01855750dp-1, 0x1.15c5787ef69aep-5,   // X = 14.5
    0x1.fe5a858c91b2cp-1, 0x1.0ccb363781cdep-5,   // X = 15.0
    0x1.fe746eb97a4dbp-1, 0x1.045f0c30e93fep-5,   // X = 15.5
    0x1.fe8c0b4ce9ae7p-1, 0x1.f8e8abc9fd0c3p-6,   // X = 16.0
    0x1.fea19e725392ep-1, 0x1.e9ffc0449aeccp-6,   // X = 16.5
    0x1.feb562125b774p-1, 0x1.dbef6c82494c4p-6,   // X = 17.0
    0x1.fec7884ea8538p-1, 0x1.cea5eee383b4ep-6,   // X = 17.5
    0x1.fed83cb8dc779p-1, 0x1.c213655cda2f4p-6,   // X = 18.0
    0x1.fee7a5528d30ep-1, 0x1.b629904d74ebbp-6,   // X = 18.5
    0x1.fef5e36108a68p-1, 0x1.aadb9e66c6123p-6,   // X = 19.0
    0x1.ff03141d653f7p-1, 0x1.a01e001fef788p-6,   // X = 19.5
    0x1.ff0f51478d634p-1, 0x1.95e64177f05c5p-6,   // X = 20.0
    0x1.ff1ab1a199d60p-1, 0x1.8c2ae903735a8p-6,   // X = 20.5
    0x1.ff254957baf15p-1, 0x1.82e35b7151bf6p-6,   // X = 21.0
    0x1.ff2f2a581aba9p-1, 0x1.7a07c2d61478dp-6,   // X = 21.5
    0x1.ff38649d795a2p-1, 0x1.7190f92cce48bp-6,   // X = 22.0
    0x1.ff41066ec0382p-1, 0x1.6978759418d3dp-6,   // X = 22.5
    0x1.ff491c955e17ep-1, 0x1.61b83be1ecffep-6,   // X = 23.0
    0x1.ff50b28be9ecdp-1, 0x1.5a4ace39649a8p-6,   // X = 23.5
    0x1.ff57d2a64630cp-1, 0x1.532b205ae4039p-6,   // X = 24.0
    0x1.ff5e863447bb9p-1, 0x1.4c548c724508ap-6,   // X = 24.5
    0x1.ff64d59fb6b64p-1, 0x1.45c2c92fd14d8p-6,   // X = 25.0
    0x1.ff6ac8865c28bp-1, 0x1.3f71e10084885p-6,   // X = 25.5
    0x1.ff7065d0b121fp-1, 0x1.395e2a4075928p-6,   // X = 26.0
    0x1.ff75b3c5ac489p-1, 0x1.33844047a2bfcp-6,   // X = 26.5
    0x1.ff7ab81c16b95p-1, 0x1.2de0fd35e0cb2p-6,   // X = 27.0
    0x1.ff7f7809c0a44p-1, 0x1.2871746679d3ep-6,   // X = 27.5
    0x1.ff83f850e0776p-1, 0x1.2332ed774224bp-6,   // X = 28.0
    0x1.ff883d4bdc0a4p-1, 0x1.1e22dfd1a3f24p-6,   // X = 28.5
    0x1.ff8c4af7b1c91p-1, 0x1.193eeea676818p-6,   // X = 29.0
    0x1.ff9024fd2feddp-1, 0x1.1484e54f711a5p-6,   // X = 29.5
    0x1.ff93ceb9212e6p-1, 0x1.0ff2b40abcd23p-6,   // X = 30.0
    0x1.ff974b4390ac1p-1, 0x1.0b866d069d120p-6,   // X = 30.5
    0x1.ff9a9d764232cp-1, 0x1.073e41b467624p-6,   // X = 31.0
    0x1.ff9dc7f277d4ap-1, 0x1.0318805b17739p-6,   // X = 31.5
    0x1.ffa0cd261a86fp-1, 0x1.fe2723c5766b4p-7,   // X = 32.0
    0x1.ffa3af50587d0p-1, 0x1.f65befa58353ap-7,   // X = 32.5
    0x1.ffa67085c9862p-1, 0x1.eecc94fbd555dp-7,   // X = 33.0
    0x1.ffa912b427947p-1, 0x1.e7766eae64211p-7,   // X = 33.5
    0x1.ffab97a5a7c0fp-1, 0x1.e056fed731686p-7,   // X = 34.0
    0x1.ffae0103fe932p-1, 0x1.d96bebfa49848p-7,   // X = 34.5
    0x1.ffb0505b18f7cp-1, 0x1.d2b2fe77b5956p-7,   // X = 35.0
    0x1.ffb2871b922b7p-1, 0x1.cc2a1e33987c4p-7,   // X = 35.5
    0x1.ffb4a69ceddacp-1, 0x1.c5cf506f50465p-7,   // X = 36.0
    0x1.ffb6b01f9cdb8p-1, 0x1.bfa0b5cf02a3fp-7,   // X = 36.5
    0x1.ffb8a4ced2213p-1, 0x1.b99c88877757bp-7,   // X = 37.0
    0x1.ffba85c22ce51p-1, 0x1.b3c11ab0914bdp-7,   // X = 37.5
    0x1.ffbc53ff3c68dp-1, 0x1.ae0cd4b918120p-7,   // X = 38.0
    0x1.ffbe107ae1393p-1, 0x1.a87e33f8d9954p-7,   // X = 38.5
    0x1.ffbfbc1a8f65cp-1, 0x1.a313c95e7815ap-7,   // X = 39.0
    0x1.ffc157b574c1bp-1, 0x1.9dcc38367c58ap-7,   // X = 39.5
    0x1.ffc2e41585e8dp-1, 0x1.98a6350980556p-7,   // X = 40.0
};

}  // namespace drt
