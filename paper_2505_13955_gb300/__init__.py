"""GB300-native parallel-beam filtered backprojection (placeholder; filled in below)."""
