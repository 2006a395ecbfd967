"""GB300-native rigid multiblob mobility solver (wall-corrected RPY)."""
